"""The library's integer-pipe FP64 <-> FP32 conversions against the
hardware conversion, bit for bit (round to nearest even, ties, the edges of
the binary32 range, subnormal results, infinities and NaN)."""
import ctypes as C

import numpy as np
import pytest

from paper_2603_19764_b300 import build, sph

pytestmark = pytest.mark.gpu


def test_conversions_match_hardware():
    import torch
    build.build()
    rng = np.random.default_rng(21)
    f32 = np.finfo(np.float32)
    vals = [rng.normal(0, 1, 200000),
            rng.normal(0, 1, 20000) * 10.0 ** rng.integers(-45, 39, 20000),
            np.exp(rng.uniform(-110, 110, 20000)) * rng.choice([-1, 1], 20000)]
    # exact ties between two floats and their neighbours
    base = rng.normal(0, 1, 5000).astype(np.float32).astype(np.float64)
    ulp = np.spacing(base.astype(np.float32)).astype(np.float64)
    vals += [base + 0.5 * ulp, base - 0.5 * ulp, base + 0.5 * ulp * (1 + 2.0 ** -30)]
    edges = [0.0, -0.0, np.inf, -np.inf, np.nan, f32.max, -f32.max, float(f32.max) * (1 + 2 ** -25),
             float(f32.max) * (1 + 2 ** -24), f32.tiny, f32.tiny / 2, f32.tiny * (1 - 2 ** -30),
             1e-45, 1e-46, 1e300, -1e300, 5e-324, 2.0 ** 127, 2.0 ** -126, 2.0 ** -149,
             1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, 1.0 - 2.0 ** -25]
    vals.append(np.array(edges, np.float64))
    x = torch.as_tensor(np.concatenate(vals)).cuda()
    bad = C.c_int64(-1)
    s = torch.cuda.current_stream().cuda_stream
    rc = sph.lib().sph_check_conversions(C.c_void_p(x.data_ptr()), x.numel(), C.byref(bad),
                                         C.c_void_p(s))
    assert rc == sph.SPH_OK
    assert bad.value == 0
