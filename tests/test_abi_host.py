"""CPU-only checks of the C ABI library: it loads, exports every symbol that
include/chase.h declares, and its host-side arithmetic (Alg. 5 CondEst,
degreeOpt) takes the same decisions as the oracle, bit for bit, on identical
inputs. No GPU call is made here."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import chase_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def _declared_symbols():
    names = set()
    for h in HEADERS:
        txt = open(h).read()
        names |= set(re.findall(r"CHASE_API\s+[\w\s\*]*?\b(chase_\w+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def pkg():
    import paper_2309_15595_gb300 as p
    return p


def test_library_exports_every_declared_symbol(pkg):
    declared = _declared_symbols()
    assert "chase_solve" in declared and "chase_filter" in declared
    lib = ctypes.CDLL(pkg._lib.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    # the binding wraps exactly the declared set
    assert set(pkg._lib.SIGNATURES) == set(declared)


def test_status_strings_and_defaults(pkg):
    assert pkg.chase_status_string(0) == "CHASE_OK"
    assert pkg.chase_status_string(6) == "CHASE_ERR_NOT_CONVERGED"
    p = pkg.default_params(512, 40, 20)
    assert (p.deg_init, p.deg_max, p.tol, p.lanczos_steps, p.lanczos_vecs) == (20, 36, 1e-10, 25, 4)


def test_create_rejects_invalid_params_without_gpu(pkg):
    h = ctypes.c_void_p()
    bad = pkg.default_params(64, 60, 10)  # nev + nex > N
    assert pkg.LIB.chase_create(ctypes.byref(bad), None, ctypes.byref(h)) == 1
    bad = pkg.default_params(64, 8, 4, deg_init=7)  # odd initial degree
    assert pkg.LIB.chase_create(ctypes.byref(bad), None, ctypes.byref(h)) == 1


def test_cond_est_matches_oracle_bitwise(pkg):
    rng = np.random.default_rng(0)
    for _ in range(200):
        n = int(rng.integers(2, 40))
        locked = int(rng.integers(0, n))
        c, e = rng.uniform(-1, 5), rng.uniform(0.1, 4)
        ritz = np.sort(rng.uniform(c - 3 * e, c + e, n))
        degs = np.sort(2 * rng.integers(1, 19, n)).astype(np.int32)
        assert pkg.chase_cond_est(ritz, degs, locked, c, e) == O.cond_est(ritz, c, e, degs, locked)


def test_degree_opt_matches_oracle_bitwise(pkg):
    rng = np.random.default_rng(1)
    for _ in range(100):
        n = int(rng.integers(1, 60))
        c, e = rng.uniform(-1, 5), rng.uniform(0.1, 4)
        ritz = rng.uniform(c - 2 * e, c + 0.5 * e, n)
        tol_abs = 10 ** rng.uniform(-12, -8)
        resid = tol_abs * 10 ** rng.uniform(-2, 12, n)
        got = pkg.chase_degree_opt(resid, ritz, c, e, tol_abs, 36, 2)
        ref = O.degree_opt(resid, ritz, c, e, tol_abs, 36, 2)
        assert np.array_equal(got, ref)


def test_new_entry_points_reject_invalid_arguments_without_gpu(pkg):
    # argument checks run before any CUDA call: null contexts and pointers,
    # negative counts are refused; an empty batch is a no-op
    L = pkg.LIB
    INVALID = 1
    status = (ctypes.c_int32 * 1)()
    assert L.chase_solve_batch(-1, None, None, None, None, None, None, None, None, None, None,
                               status, 0) == INVALID
    assert L.chase_solve_batch(0, None, None, None, None, None, None, None, None, None, None,
                               None, 0) == 0
    assert L.chase_solve_batch(1, None, None, None, None, None, None, None, None, None, None,
                               status, 0) == INVALID
    assert L.chase_filter_vjp(None, None, 1, None, 1, 1, 2, 1.0, 1.0, -1.0, None, 1, None, 1,
                              None, 1, 0) == INVALID
    it = ctypes.c_int32(0)
    assert L.chase_eig_vjp(None, None, 1, None, 1, None, 1, 1, None, None, 1, None, 1, 1e-10,
                           100, ctypes.byref(it)) == INVALID


def _prototypes():
    """name -> number of parameters of every CHASE_API function in include/*.h"""
    out = {}
    for h in HEADERS:
        txt = re.sub(r"/\*.*?\*/", " ", open(h).read(), flags=re.S)
        for name, params in re.findall(r"CHASE_API\s+[\w\s\*]*?\b(chase_\w+)\s*\(([^;]*?)\)\s*;",
                                       txt, flags=re.S):
            params = params.strip()
            out[name] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_argument_counts_match_the_header(pkg):
    protos = _prototypes()
    assert set(protos) == set(pkg._lib.SIGNATURES)
    for name, (_, args) in pkg._lib.SIGNATURES.items():
        assert len(args) == protos[name], name


def test_binding_structs_match_the_header_layout(pkg, tmp_path):
    """sizeof and every field offset of chase_params and chase_stats as the C
    compiler lays them out from include/chase.h, against the ctypes mirrors."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"chase_params": pkg._lib.ChaseParams, "chase_stats": pkg._lib.ChaseStats}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "chase.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True,
                               text=True).stdout.splitlines():
        cname, key, val = line.split()
        got[(cname, key)] = int(val)
    for cname, cls in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
