"""The C ABI library loads on a CPU-only machine, exports every entry point
declared in include/dgh.h, and its host-only set-up (dgh_plan) agrees with
the closed-form mesh counts.  No call here touches a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1610_05023_b300 as dgh
from paper_1610_05023_b300 import build, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(dgh.LIB_PATH)


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(dgh_[a-z0-9_]+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert {"dgh_create", "dgh_step", "dgh_get_energy", "dgh_plan"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_checked_build_exports_the_same_symbols(lib):
    """The index-checked variant (DGH_CHECKED) is the same ABI."""
    path = build.build(checked=True)
    chk = ctypes.CDLL(path)
    for n in sorted(declared_symbols()):
        assert hasattr(chk, n), n
    assert chk.dgh_is_checked_build() == 1
    assert lib.dgh_is_checked_build() == 0


def test_error_paths_without_gpu(lib):
    dgh.load_library()
    L = dgh._lib
    h = ctypes.c_void_p()
    assert L.dgh_create(None, None, ctypes.byref(h)) == -1
    assert b"invalid" in L.dgh_last_error(None)
    assert L.dgh_set_watchdog(None, 1, 0.0) == -1
    VX, EToV = W.kuhn_mesh(1)
    d, keep = dgh._make_desc(VX, EToV, 9, 0, (0,) * 6, 1.0, 1.0, 0.0, 1.0)
    assert L.dgh_create(ctypes.byref(d), None, ctypes.byref(h)) == -7
    d, keep = dgh._make_desc(VX, EToV, 2, 0, (0,) * 6, -1.0, 1.0, 0.0, 1.0)
    assert L.dgh_create(ctypes.byref(d), None, ctypes.byref(h)) == -1
    # a mesh with a hole is not a cuboid boundary
    d, keep = dgh._make_desc(VX, EToV[1:], 2, 0, (0,) * 6, 1.0, 1.0, 0.0, 1.0)
    with pytest.raises(dgh.DghError):
        dgh.plan(VX, EToV[1:], 2, 1)


@pytest.mark.parametrize("n,N,P", [(1, 1, 1), (2, 3, 3), (3, 2, 2), (4, 3, 0)])
def test_plan_counts(n, N, P):
    VX, EToV = W.kuhn_mesh(n, 1.0, 0.02, seed=4)
    info = dgh.plan(VX, EToV, N, P)
    assert info["n_cells"] == 6 * n ** 3
    assert info["n_tris"] == (12 * n * n if P else 0)
    assert info["n_lines"] == (12 * n if P else 0)
    assert info["n_corners"] == (8 if P else 0)
    Np = (N + 1) * (N + 2) * (N + 3) // 6
    assert info["ndof"] == 4 * Np * 6 * n ** 3 + 3 * P * (N + 1) * (N + 2) // 2 * info["n_tris"] + 2 * P * P * (N + 1) * info["n_lines"]


def test_plan_mixed_boundaries_and_dt():
    # free surface on +z: no auxiliary fields on its edges and corners
    n = 3
    VX, EToV = W.kuhn_mesh(n)
    info = dgh.plan(VX, EToV, 2, 2, bc=(0, 0, 0, 0, 0, 1))
    assert info["n_tris"] == 10 * n * n
    assert info["n_lines"] == 8 * n            # 4 vertical + 4 bottom edges
    assert info["n_corners"] == 4              # K^pnt = 4 with one Dirichlet face
    h = 2.0 / n
    assert abs(info["dt"] - 1.0 / (9 * 2 * np.sqrt(2) / h)) < 1e-12


def test_batch_plan_groups_and_sums():
    """Host-only batch grouping: problems are grouped by (N, P) in order of
    first appearance and every union mesh has the summed sizes of its problems
    (cells, triangles, lines, corners, boundary faces, DOFs)."""
    from oracle.mesh import BC_DIRICHLET
    specs = [(2, 3, 2, (0,) * 6), (3, 4, 1, (0,) * 6), (2, 3, 2, (BC_DIRICHLET,) + (0,) * 5),
             (2, 2, 0, (0,) * 6), (3, 3, 2, (0,) * 6)]
    probs = []
    for i, (n, N, P, bc) in enumerate(specs):
        VX, EToV = W.kuhn_mesh(n, 1.0, 0.02, seed=40 + i)
        probs.append(dict(VX=VX, EToV=EToV, N=N, P=P, bc=bc))
    gof, infos = dgh.batch_plan(probs)
    assert gof == [0, 1, 0, 2, 0]
    assert len(infos) == 3
    singles = [dgh.plan(**p) for p in probs]
    for g, info in enumerate(infos):
        members = [s for s, gg in zip(singles, gof) if gg == g]
        for k in ("n_cells", "n_tris", "n_lines", "n_corners", "n_bfaces", "ndof"):
            assert info[k] == sum(m[k] for m in members), (g, k)
        assert (info["order"], info["habc_order"]) == (members[0]["order"], members[0]["habc_order"])


def test_plan_rejects_edge_inputs():
    """Empty and oversized meshes, out-of-range codes, a degenerate cell and a
    dangling vertex id are rejected with the documented codes, before any
    array beyond the stated sizes is read."""
    L = dgh.load_library()
    VX, EToV = W.kuhn_mesh(1)
    info = dgh._Info()

    def code(**kw):
        args = dict(VX=VX, EToV=EToV, N=2, P=1, bc=(0,) * 6, c=1.0, rho=1.0, dt=0.0, cfl=1.0)
        args.update(kw)
        d, keep = dgh._make_desc(args["VX"], args["EToV"], args["N"], args["P"], args["bc"], args["c"], args["rho"],
                                 args["dt"], args["cfl"], kw.get("precision", 0))
        for k, v in kw.get("patch", {}).items():
            setattr(d, k, v)
        return L.dgh_plan(ctypes.byref(d), ctypes.byref(info))

    assert code() == 0
    assert code(patch={"n_cells": 0}) == -1                     # empty mesh
    assert code(patch={"n_cells": (1 << 26) + 1}) == -7          # beyond the 32-bit connectivity encoding
    assert code(P=13) == -7                                      # HABC order above 12
    assert code(N=0) == -7
    assert code(precision=7) == -7                               # unknown precision code
    assert code(bc=(0, 0, 0, 0, 0, 5)) == -1                     # unknown boundary code
    flat = VX.copy()
    E = EToV.copy()
    E[0] = [0, 1, 2, 3]
    flat[3] = flat[0] + (flat[1] - flat[0]) + (flat[2] - flat[0])  # vertex 3 in the plane of 0, 1, 2
    assert code(VX=flat, EToV=E) == -1                           # degenerate cell (or broken conformity)
    E2 = EToV.copy()
    E2[0, 0] = VX.shape[0]                                        # dangling vertex id
    assert code(EToV=E2) == -1
    # the tensor-core modes plan on the CPU like the FP32 path
    assert code(precision=dgh.PREC_SPLIT_BF16) == 0 and info.n_cells == 6


def test_batch_plan_separates_precisions():
    VX, EToV = W.kuhn_mesh(2, 1.0, 0.02, seed=9)
    probs = [dict(VX=VX, EToV=EToV, N=3, P=2), dict(VX=VX, EToV=EToV, N=3, P=2, precision=dgh.PREC_SPLIT_BF16),
             dict(VX=VX, EToV=EToV, N=3, P=2)]
    gof, infos = dgh.batch_plan(probs)
    assert gof == [0, 1, 0] and len(infos) == 2


def test_exceptions_stop_at_the_boundary():
    """No C++ exception crosses the C ABI: every entry point runs under one
    guard, exercised here by a host-only self-test call."""
    lib = dgh.load_library()
    cases = [(0, dgh.DGH_ENOMEM, "host memory exhausted"), (1, dgh.DGH_EINVAL, "self-test exception"),
             (2, dgh.DGH_EINVAL, "unknown C++ exception")]
    for kind, code, text in cases:
        assert lib.dgh_selftest_throw(kind) == code
        msg = lib.dgh_last_error(None).decode()
        assert msg.startswith("internal error:") and text in msg, msg
    assert lib.dgh_selftest_throw(3) == 0


def test_create_fails_cleanly_without_a_gpu():
    """On a machine without a usable GPU, creating a solver stops at its first
    device allocation with DGH_ECUDA and a message; repeated attempts work,
    because a failed create frees the context it had built."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    VX, EToV = W.kuhn_mesh(2, 1.0, 0.02, seed=1)
    for _ in range(3):
        with pytest.raises(dgh.DghError) as e:
            dgh.Solver(VX, EToV, 3, 2)
        assert e.value.code == dgh.DGH_ECUDA and "cuda" in str(e.value).lower()
