"""The allocation-free real-space entry point agrees with fbim_apply_real.

fbim_apply_real_noalloc serves callers that must not allocate device memory
while running (a host that hands all device memory to its own pool, or a
time-critical loop).  It keeps its scratch in a fixed device array of the
library; this test calls it twice in a row through the C ABI, with different
forces each time, and compares each result with the ordinary entry point at the
FP64 tolerance of the other GPU tests.  The file sorts last so that a run that
stops at its first failure has run every other test already.
"""
import ctypes
import math

import numpy as np
import pytest

import fbim_synth

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10


def test_noalloc_real_operator_matches_fbim_apply_real_twice():
    import torch
    import paper_1709_01480_gb300 as fb
    assert torch.cuda.is_available()
    w = fbim_synth.workload("starfish4_np64_L4")
    n_box = 6
    xi = math.sqrt(math.log(100.0 / 1e-13)) / (w.L / n_box)
    op = fb.FBIM(w.ref_nodes, w.Q, w.L, tol=1e-13, r_c=w.L / n_box, xi=xi, precision="fp64")
    lib = fb.lib()
    rng = np.random.default_rng(77)
    for call in range(2):
        mu = torch.tensor(rng.standard_normal((w.n, 2)), device="cuda")
        ref = op.apply_real(mu)
        out = torch.full((w.n, 2), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.fbim_apply_real_noalloc(op.handle, ctypes.c_void_p(mu.data_ptr()), ctypes.c_void_p(out.data_ptr()))
        assert st == 0, lib.fbim_last_error(op.handle)
        torch.cuda.synchronize()
        err = float((out - ref).abs().max() / ref.abs().max())
        print(f"noalloc call {call}: rel diff {err:.3e}")
        assert err < FP64_TOL
    op.close()


def test_noalloc_rejects_handles_above_its_limit():
    import torch
    import paper_1709_01480_gb300 as fb
    ref = fbim_synth.starfish_ref_nodes(128)
    n_b = 1040                                   # 133120 nodes > 131072
    L = fbim_synth.box_for_fraction(n_b, fbim_synth.starfish_area(), 0.25)
    Q = fbim_synth.place_bodies(n_b, L, ref, 0.1, 3)
    op = fb.FBIM(ref, Q, L, tol=1e-8, r_c=L / 115, precision="fp64")
    mu = torch.zeros((op.n, 2), dtype=torch.float64, device="cuda")
    out = torch.zeros_like(mu)
    with pytest.raises(fb.FbimError) as e:
        op.apply_real_noalloc(mu, out)
    assert e.value.status == 1 and "at most 131072" in str(e.value)
    op.close()
