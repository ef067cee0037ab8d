"""The allocation-free real-space entry point agrees with fbim_apply_real.

fbim_apply_real_noalloc serves callers that must not allocate device memory
while running (a host that hands all device memory to its own pool, or a
time-critical loop).  It keeps its scratch in a fixed device array of the
library; this test calls it twice in a row through the C ABI, with different
forces each time, and compares each result with the ordinary entry point at the
FP64 tolerance of the other GPU tests.  The file sorts last so that a run that
stops at its first failure has run every other test already.

Under CUDA's lazy module loading a kernel's module is loaded, and device memory
allocated for it, at its first use; fbim_setup therefore loads the entry point's
kernels ahead of time.  A child process with CUDA_MODULE_LOADING=LAZY checks that
the device's free memory is the same before and after the entry point's first two
calls.
"""
import ctypes
import json
import math
import os
import subprocess
import sys

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


_FREE_MEMORY_PROBE = r"""
import ctypes, json, math, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import torch
import fbim_synth
import paper_1709_01480_gb300 as fb
w = fbim_synth.workload("starfish4_np64_L4")
xi = math.sqrt(math.log(100.0 / 1e-13)) / (w.L / 6)
op = fb.FBIM(w.ref_nodes, w.Q, w.L, tol=1e-13, r_c=w.L / 6, xi=xi, precision="fp32")
mu = torch.tensor(np.random.default_rng(3).standard_normal((w.n, 2)), device="cuda")
out = torch.empty_like(mu)
ref = op.apply_real(mu).clone()
torch.cuda.synchronize()
lib = fb.lib()
free0 = torch.cuda.mem_get_info()[0]
codes = [lib.fbim_apply_real_noalloc(op.handle, ctypes.c_void_p(mu.data_ptr()), ctypes.c_void_p(out.data_ptr()))
         for _ in range(2)]
torch.cuda.synchronize()
free1 = torch.cuda.mem_get_info()[0]
print(json.dumps({"codes": codes, "free_before": free0, "free_after": free1,
                  "rel_diff_fp32_handle": float((out - ref).abs().max() / ref.abs().max())}))
op.close()
"""


def test_noalloc_first_calls_allocate_nothing_under_lazy_loading():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CUDA_MODULE_LOADING="LAZY")
    r = subprocess.run([sys.executable, "-c", _FREE_MEMORY_PROBE, root], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip().splitlines()[-1])
    print(d)
    assert d["codes"] == [0, 0]
    assert d["free_after"] == d["free_before"], d
    # an FP32 handle's real-space operator is FP32: agreement to its rounding
    assert d["rel_diff_fp32_handle"] < 1e-5


def test_noalloc_wrapper_rejects_tensors_it_cannot_use():
    import torch
    import paper_1709_01480_gb300 as fb
    w = fbim_synth.workload("starfish4_np64_L4")
    op = fb.FBIM(w.ref_nodes, w.Q, w.L, tol=1e-10, r_c=w.L / 6, precision="fp64")
    good = torch.zeros((w.n, 2), dtype=torch.float64, device="cuda")
    bad = [torch.zeros((w.n, 2), dtype=torch.float32, device="cuda"),        # wrong dtype
           torch.zeros((w.n - 1, 2), dtype=torch.float64, device="cuda"),    # wrong shape
           torch.zeros((2, w.n), dtype=torch.float64, device="cuda").t(),    # not contiguous
           torch.zeros((w.n, 2), dtype=torch.float64)]                       # host memory
    for b in bad:
        for args in ((b, good), (good, b)):
            with pytest.raises(fb.FbimError) as e:
                op.apply_real_noalloc(*args)
            assert e.value.status == 1
    op.apply_real_noalloc(good, torch.empty_like(good))
    op.close()
