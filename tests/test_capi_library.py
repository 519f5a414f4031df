"""The C ABI library without a GPU: it builds, loads, exports exactly the
entry points include/se2n.h declares, and its host-only functions behave.
No device computation is started here."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "se2n.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"SE2N_API\s+[\w\s\*]+?\b(se2n_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1304_2062_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["se2n_plan_create", "se2n_plan_destroy", "se2n_orient", "se2n_lift", "se2n_forward",
                     "se2n_diffuse", "se2n_inverse", "se2n_mix", "se2n_dr_grow", "se2n_project", "se2n_inpaint",
                     "se2n_inpaint_host", "se2n_params_from_paper", "se2n_status_string"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_only_the_c_abi_is_exported(lib):
    from paper_1304_2062_gb300 import build
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = sorted(ln.split()[-1] for ln in out.splitlines() if ln.strip())
    assert exported == _declared()


def test_status_strings(lib):
    lib.se2n_status_string.restype = ctypes.c_char_p
    for s in range(7):
        assert lib.se2n_status_string(s).decode().startswith("SE2N")
    assert b"unknown" in lib.se2n_status_string(99)


def test_params_from_paper_matches_oracle(lib):
    f = lib.se2n_params_from_paper
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                  ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    b, t = ctypes.c_double(), ctypes.c_double()
    for alpha, T, M, N in [(2.0, 0.8, 256, 30), (0.33, 6.0, 256, 30), (0.25, 0.15, 512, 32)]:
        assert f(alpha, T, M, N, ctypes.byref(b), ctypes.byref(t)) == 0
        ob, oT = oracle.params_from_paper(alpha, T, M, N)
        assert abs(b.value - ob) <= 1e-15 * ob and abs(t.value - oT) <= 1e-12 * oT
    assert f(-1.0, 1.0, 256, 30, ctypes.byref(b), ctypes.byref(t)) == 1
    assert f(1.0, 1.0, 256, 30, None, ctypes.byref(t)) == 1


def test_params_default(lib):
    from paper_1304_2062_gb300.se2n import se2n_params
    p = se2n_params()
    p.reinject = p.full_spectrum = p.dynamic = 7      # the C side must reach the last field
    lib.se2n_params_default.argtypes = [ctypes.POINTER(se2n_params)]
    assert lib.se2n_params_default(ctypes.byref(p)) == 0
    assert (p.N, p.steps, p.rounds, p.proj, p.final_mix) == (32, 100, 1, 0, 0)
    assert (p.reinject, p.full_spectrum, p.dynamic) == (0, 0, 0)
    assert (p.beta, p.eps, p.sigma_smooth, p.flat_tol) == (0.25, 0.5, 1.0, 1e-4)
    assert lib.se2n_params_default(None) == 1


def test_plan_arguments_are_checked_before_any_device_work(lib):
    """Invalid sizes are rejected on the host (EINVAL / EUNSUPPORTED)
    whether or not a GPU is present; with valid sizes and no GPU the call
    fails cleanly with ECUDA instead of crashing."""
    lib.se2n_plan_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_void_p]
    h = ctypes.c_void_p()
    assert lib.se2n_plan_create(ctypes.byref(h), 7, 8, 16, 0, None) == 1
    assert lib.se2n_plan_create(ctypes.byref(h), 8, 8, 2, 0, None) == 1
    assert lib.se2n_plan_create(ctypes.byref(h), 8, 8, 16, 2, None) == 1
    assert lib.se2n_plan_create(ctypes.byref(h), 8, 8, 10, 0, None) == 5
    assert lib.se2n_plan_create(None, 8, 8, 16, 0, None) == 1
    import torch
    if not torch.cuda.is_available():
        assert lib.se2n_plan_create(ctypes.byref(h), 8, 8, 16, 0, None) == 3
        assert h.value is None
    # a NULL plan is rejected everywhere
    assert lib.se2n_plan_destroy(None) == 0
    assert lib.se2n_forward(None, None) == 1


def test_python_binding_loads_and_names_match_the_c_abi():
    from paper_1304_2062_gb300 import se2n
    for name in _declared():
        assert callable(getattr(se2n, name)), name


def _run_chain(ops, in_r):
    """Exponents of P and R after the program (P = D_1, R empty at the start)."""
    p, r = 1, 0
    for o in ops:
        if o == 0:
            p = 2 * p
        elif o == 1:
            assert r > 0
            p = 2 * r
        elif o == 2:
            assert r > 0
            r = r + p
        else:
            assert o == 3
            r = p
    return r if in_r else p


def _fewest_products(S):
    """Brute force: breadth-first over the exponent pairs (p, r) of every
    two-matrix program, products cost 1 and copies 0."""
    from collections import deque
    dist = {(1, 0): 0}
    q = deque([(1, 0)])
    while q:
        p, r = q.popleft()
        d = dist[(p, r)]
        if p == S or r == S:
            return d
        moves = [((p, p), 0)] if r != p else []
        if 2 * p <= S:
            moves.append(((2 * p, r), 1))
        if r and 2 * r <= S:
            moves.append(((2 * r, r), 1))
        if r and p + r <= S:
            moves.append(((p, p + r), 1))
        for st, c in moves:
            if st not in dist or dist[st] > d + c:
                dist[st] = d + c
                (q.appendleft if c == 0 else q.append)(st)
    raise AssertionError(S)


def test_powering_program_reaches_S_with_the_fewest_products():
    """The propagator's powering program (D_m = M^m - I over two matrices):
    it reaches S, takes no more products than binary powering, and as few as
    a brute-force search over all two-matrix programs."""
    from paper_1304_2062_gb300 import se2n
    for S in list(range(1, 65)) + [100, 127, 255, 500, 1000, 4095, 4096, 4097, 100000, 2 ** 31 - 1]:
        ops, in_r = se2n.se2n_prop_chain(S)
        assert _run_chain(ops, in_r) == S
        products = sum(o != 3 for o in ops)
        assert products <= S.bit_length() - 1 + bin(S).count("1") - 1
        if S <= 64 or S == 500:
            assert products == _fewest_products(S), S
    assert sum(o != 3 for o in se2n.se2n_prop_chain(500)[0]) == 11


def test_powering_program_arguments_are_checked(lib):
    f = lib.se2n_prop_chain
    f.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                  ctypes.POINTER(ctypes.c_int)]
    buf = (ctypes.c_ubyte * 64)()
    n, r = ctypes.c_int(), ctypes.c_int()
    assert f(0, buf, 64, ctypes.byref(n), ctypes.byref(r)) == 1
    assert f(500, None, 64, ctypes.byref(n), ctypes.byref(r)) == 1
    assert f(500, buf, 64, None, ctypes.byref(r)) == 1
    assert f(500, buf, 5, ctypes.byref(n), ctypes.byref(r)) == 1
    assert f(1, buf, 0, ctypes.byref(n), ctypes.byref(r)) == 0 and n.value == 0 and r.value == 0
