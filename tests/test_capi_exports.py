"""The C ABI library builds for sm_103a, loads, and exports every entry point
declared in include/hfmm.h with the binding's signature table covering them
all.  No compute calls: this runs without a GPU."""
import ctypes
import numpy as np
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, re.M):
            name = m.group(1)
            if name not in ("defined",):
                names.append(name)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    from paper_1608_02461_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fmm_build_tree", "fmm_apply", "fmm_precond_apply", "gmres_solve",
                     "fmm_destroy_tree", "fmm_get_stats", "hfmm_error_string", "hfmm_fdm_apply"):
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    for name in declared_functions():
        assert hasattr(built_lib, name), name


def test_binding_covers_every_symbol():
    from paper_1608_02461_gb300 import hfmm
    assert set(declared_functions()) <= set(hfmm.SIGNATURES)


def test_error_strings(built_lib):
    f = built_lib.hfmm_error_string
    f.restype = ctypes.c_char_p
    f.argtypes = [ctypes.c_int]
    assert f(0) == b"ok"
    assert b"argument" in f(-1)
    assert b"converge" in f(-5)


def test_invalid_arguments_rejected_without_gpu(built_lib):
    """Argument checks happen before any device work."""
    from paper_1608_02461_gb300 import hfmm
    L = hfmm.lib()
    out = ctypes.c_void_p()
    bad = [hfmm.hfmm_params(0, 0.4, 64, 4.0, 0), hfmm.hfmm_params(4, 0.9, 64, 4.0, 0),
           hfmm.hfmm_params(4, 0.4, 0, 4.0, 0), hfmm.hfmm_params(4, 0.4, 64, -1.0, 0),
           hfmm.hfmm_params(4, 0.4, 64, 4.0, 7), hfmm.hfmm_params(40, 0.4, 64, 4.0, 0)]
    for prm in bad:
        st = L.fmm_build_tree(16, None, 0, None, 0, ctypes.byref(prm), None, ctypes.byref(out))
        assert st == hfmm.HFMM_ERR_INVALID_ARG
        assert not out.value
    st = L.fmm_build_tree(1, None, 0, None, 0, ctypes.byref(hfmm.hfmm_params(4, 0.4, 64, 4.0, 0)),
                          None, ctypes.byref(out))
    assert st == hfmm.HFMM_ERR_INVALID_ARG
    assert L.fmm_apply(None, 1, 1, None, None, None, None, 0, None) == hfmm.HFMM_ERR_INVALID_ARG
    assert L.gmres_solve(None, None, None, None, None, None) == hfmm.HFMM_ERR_INVALID_ARG
    assert L.bicgstab_solve(None, None, None, None, None, None) == hfmm.HFMM_ERR_INVALID_ARG
    assert L.fmm_precond_apply(None, None, None, 1e-2, 20, 20, None, None) == hfmm.HFMM_ERR_INVALID_ARG
    assert L.fmm_autotune(None, None) == hfmm.HFMM_ERR_INVALID_ARG
    assert L.fmm_use_graphs(None, 1) == hfmm.HFMM_ERR_INVALID_ARG
    assert L.fmm_apply(None, hfmm.SET_BND, 1, None, None, None, None, hfmm.DLP, None) == hfmm.HFMM_ERR_INVALID_ARG
    assert L.hfmm_dirichlet_rhs(None, None, None, None, None) == hfmm.HFMM_ERR_INVALID_ARG
    assert L.bem_solve_dirichlet(None, None, None, None, 1e-2, 20, 20, None, None) == hfmm.HFMM_ERR_INVALID_ARG
    assert L.fmm_set_inner_order(None, 4, None) == hfmm.HFMM_ERR_INVALID_ARG
    assert L.fmm_grad_k(None, None, None, None, None) == hfmm.HFMM_ERR_INVALID_ARG
    assert L.hfmm_solve_grad_k(None, None, None, None, None) == hfmm.HFMM_ERR_INVALID_ARG


def test_binding_prototypes_match_header_arity():
    """Every prototype of the binding has as many arguments as the header's
    declaration (a mismatch would pass garbage through ctypes)."""
    import re as _re
    from paper_1608_02461_gb300 import hfmm
    src = open(os.path.join(ROOT, "include", "hfmm.h")).read()
    src = _re.sub(r"/\*.*?\*/", "", src, flags=_re.S)
    for name, (_, args) in hfmm.SIGNATURES.items():
        m = _re.search(r"\b" + name + r"\s*\(([^;]*?)\)\s*;", src, _re.S)
        assert m, name
        params = [p for p in m.group(1).split(",") if p.strip() and p.strip() != "void"]
        assert len(params) == len(args), (name, len(params), len(args))


def test_noalloc_binding_rejects_bad_arguments_before_launch():
    """direct_sum_noalloc checks dtype, shape, length, contiguity and device of
    every tensor before it calls the library (nothing here reaches a GPU)."""
    torch = pytest.importorskip("torch")
    from paper_1608_02461_gb300 import hfmm
    n_src, n_tgt = 5, 3
    good = dict(src_xyz=torch.zeros(n_src, 3, dtype=torch.float64),
                q=torch.zeros(n_src, dtype=torch.complex128),
                tgt_xyz=torch.zeros(n_tgt, 3, dtype=torch.float64),
                phi=torch.zeros(n_tgt, dtype=torch.complex128))
    assert hfmm.check_noalloc_args(**good, require_cuda=False) == (n_src, n_tgt)
    bad = [
        ("q", torch.zeros(n_src, dtype=torch.complex64)),                 # complex64 weights
        ("q", torch.zeros(n_src + 1, dtype=torch.complex128)),            # wrong length
        ("q", torch.zeros(2 * n_src, dtype=torch.complex128)[::2]),       # non-contiguous view
        ("phi", torch.zeros(n_tgt - 1, dtype=torch.complex128)),          # phi shorter than the targets
        ("phi", torch.zeros(n_tgt, dtype=torch.complex64)),
        ("src_xyz", torch.zeros(n_src, 3, dtype=torch.float32)),          # float32 coordinates
        ("src_xyz", torch.zeros(3, n_src, dtype=torch.float64).t()),      # transposed view
        ("tgt_xyz", torch.zeros(n_tgt, 2, dtype=torch.float64)),          # not (n, 3)
        ("tgt_xyz", torch.zeros(3 * n_tgt, dtype=torch.float64)),         # flat
    ]
    for name, t in bad:
        args = dict(good)
        args[name] = t
        with pytest.raises(ValueError):
            hfmm.check_noalloc_args(**args, require_cuda=False)
    # host tensors are refused before the library is called
    with pytest.raises(ValueError):
        hfmm.direct_sum_noalloc(good["src_xyz"], good["q"], good["tgt_xyz"], 1.0, good["phi"])
    # more targets than the scratch array holds
    big = hfmm.NOALLOC_MAX_TARGETS + 1
    args = dict(good, tgt_xyz=torch.zeros(big, 3, dtype=torch.float64),
                phi=torch.zeros(big, dtype=torch.complex128))
    with pytest.raises(ValueError):
        hfmm.check_noalloc_args(**args, require_cuda=False)


def test_order_for_k_rule(built_lib):
    """hfmm_order_for_k (host only): the smallest even order >= p_min with
    p >= ceil(k sqrt(3)/8) + 1.  The named workloads keep their orders; the
    batched solves that stalled at p = 4 (k >= 21.75) get 6 or 8."""
    import math
    from paper_1608_02461_gb300 import hfmm
    for k, p in [(4.0, 4), (16.0, 6), (32.0, 8), (12.0, 6)]:
        assert hfmm.order_for_k(k, p) == p
    assert hfmm.order_for_k(21.754, 4) == 6
    assert hfmm.order_for_k(26.091, 4) == 8
    assert hfmm.order_for_k(30.95, 4) == 8
    assert hfmm.order_for_k(30.84, 6) == 8
    assert hfmm.order_for_k(13.745, 4) == 4
    assert hfmm.order_for_k(0.0, 3) == 3
    for k in np.linspace(0.0, 60.0, 241):
        for pmin in (1, 4, 5, 6):
            p = hfmm.order_for_k(k, pmin)
            need = math.ceil(k * math.sqrt(3.0) / 8.0) + 1
            assert p >= pmin and p >= need
            assert p == pmin or (p % 2 == 0 and p - 2 < max(need, pmin))
    L = hfmm.lib()
    assert L.hfmm_order_for_k(-1.0, 4) == hfmm.HFMM_ERR_INVALID_ARG
    assert L.hfmm_order_for_k(float("nan"), 4) == hfmm.HFMM_ERR_INVALID_ARG
    assert L.hfmm_order_for_k(5.0, 0) == hfmm.HFMM_ERR_INVALID_ARG
    assert L.hfmm_order_for_k(200.0, 4) == hfmm.HFMM_ERR_UNSUPPORTED
