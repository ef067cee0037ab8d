"""The C-ABI library loads, exports what include/fbim.h declares, and its host logic is right.

No compute call needs a GPU here: only host-side functions are called.
"""
import math
import os
import re

import numpy as np
import pytest
from scipy.special import exp1

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    txt = open(os.path.join(ROOT, "include", "fbim.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fbim_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def fb():
    import paper_1709_01480_gb300 as fb
    return fb


def test_library_exports_every_declared_symbol(fb):
    decl = _declared_symbols()
    assert len(decl) >= 10
    for name in decl:
        assert hasattr(fb.lib(), name), name
    assert sorted(fb.EXPORTS) == decl


def test_host_e1_matches_scipy(fb):
    for z in np.concatenate([np.geomspace(1e-8, 1.0, 40), np.linspace(1.0, 40.0, 80)]):
        assert abs(fb.host_expint_e1(z) / exp1(z) - 1.0) < 5e-15


def test_host_alpert_rule_matches_oracle(fb):
    from oracle import alpert
    # the library solves in long double (80-bit on x86); the order-8 system is
    # conditioned so that its nodes carry ~1e-12 of that rounding
    for order, tol in ((4, 1e-13), (8, 1e-11)):
        v, w, a = fb.host_alpert_rule(order)
        vo, wo, ao = alpert.alpert_rule(order)
        assert a == ao
        assert np.max(np.abs(v - vo)) < tol and np.max(np.abs(w - wo)) < tol


def test_parameter_rules_reproduce_printed_xi(fb):
    # Sec. 4.2: N_box = 4 in the unit cell at tol 1e-9 gives xi ~ 20.13;
    # Sec. 4.3: N_box = 10 gives xi ~ 50.
    p = fb.choose_ewald(1.0, 0.25, 1e-9)
    assert p["n_box"] == 4 and abs(p["xi"] - 20.13) < 0.01
    p = fb.choose_ewald(1.0, 0.1, 1e-9)
    assert p["n_box"] == 10 and abs(p["xi"] - 50.3) < 0.1


def test_parameter_rules_bound_the_truncation_errors(fb):
    for L, rc, tol in ((4.0, 4.0 / 6, 1e-10), (57.98, 0.504, 1e-8), (10.0, 1.0, 1e-12)):
        p = fb.choose_ewald(L, rc, tol)
        xi, M, P = p["xi"], p["grid"], p["support"]
        assert 100 * math.exp(-(xi * p["r_c"]) ** 2) <= tol * (1 + 1e-9)
        q = (math.pi * M / L) ** 2 / (4 * xi ** 2)
        assert (1 + q) * math.exp(-q) <= tol          # Hasimoto weight of the first dropped mode
        assert P % 2 == 1 and math.exp(-math.pi * P / 2) <= tol
        assert M % 2 == 0 and 0 < p["eta_s"] < 1


def test_invalid_arguments_are_rejected(fb):
    with pytest.raises(fb.FbimError):
        fb.choose_ewald(1.0, 0.6, 1e-8)      # r_c > L/3
    with pytest.raises(fb.FbimError):
        fb.choose_ewald(1.0, 0.2, 2.0)       # tol >= 1
    # the Brownian dynamics position update checks its arguments before any CUDA call
    lib = fb.lib()
    inv = 1  # FBIM_ERR_INVALID_ARG
    fake = 4096  # never dereferenced: every call below returns before touching memory
    assert lib.fbim_bd_update(None, 3, 0.1, 0.0, None, None, None, fake) == inv      # no U
    assert lib.fbim_bd_update(None, 3, 0.1, 0.0, fake, None, None, None) == inv      # no Q
    assert lib.fbim_bd_update(None, 3, 0.1, 1.0, fake, fake, None, fake) == inv      # Up without Um
    assert lib.fbim_bd_update(None, 3, float("nan"), 0.0, fake, None, None, fake) == inv
    assert lib.fbim_bd_update(None, 1 << 40, 0.1, 0.0, fake, None, None, fake) == inv
    assert lib.fbim_bd_update(None, 0, 0.1, 0.0, fake, None, None, fake) == 0       # nothing to do
    # an unknown Brownian dynamics scheme (0 EM, 1 AB2, 2 EM without RFD) is rejected
    assert lib.fbim_bd_step(fake, 3, fake, 0.1, 1.0, 1e-3, 0, 0, None, None, None, 1e-6, 1e-6, 10, fake, 0,
                            fake, None) == inv


def test_ctypes_structs_match_the_header_layout(fb, tmp_path):
    """Every field of the binding's ctypes structs sits at the offset, and every struct
    has the size, that a C compiler gives the header's structs."""
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"fbim_params": fb.Params, "fbim_info": fb.Info, "fbim_batch_info": fb.BatchInfo}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "fbim.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'    printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_binding_checks_tensors_before_calling_the_library(fb):
    """The binding hands bare pointers to the library: a tensor of the wrong type, size,
    layout or device is refused on the host, before any library call (the handle below
    does not exist, so reaching the library would fail differently)."""
    import torch
    op = fb.FBIM.__new__(fb.FBIM)
    op.n_b, op.n_p, op.device, op._h = 2, 4, 0, None
    bad = [torch.zeros((8, 2), dtype=torch.float32),          # FP32
           torch.zeros((8, 2), dtype=torch.float64),          # host memory
           torch.zeros((2, 8), dtype=torch.float64).t(),      # not contiguous
           torch.zeros((7, 2), dtype=torch.float64)]          # wrong size
    for t in bad:
        with pytest.raises(fb.FbimError):
            op.apply_stokeslet(t)
        with pytest.raises(fb.FbimError):
            op.apply_real_noalloc(t, t)
    with pytest.raises(fb.FbimError):
        op.mobility_solve(torch.zeros((2, 3), dtype=torch.float32))
    with pytest.raises(fb.FbimError):
        op.bd_step(torch.zeros((2, 3), dtype=torch.float64), torch.zeros((2, 3), dtype=torch.float64), 1e-3)
