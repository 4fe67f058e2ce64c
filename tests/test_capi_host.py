"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function declared in include/*.h, computes node coordinates in the
documented orders, and rejects invalid arguments."""

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    import paper_2503_17535_gb300 as P
    from paper_2503_17535_gb300 import _capi
    if not os.path.exists(_capi.LIB_PATH):
        from paper_2503_17535_gb300 import build
        build.build()
    return P


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if not fn.endswith(".h"):
            continue
        txt = open(os.path.join(inc, fn)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names.update(re.findall(r"\b(hps_[a-z_]+)\s*\(", txt))
    return sorted(names)


def test_every_declared_symbol_is_exported(pkg):
    from paper_2503_17535_gb300 import _capi
    lib = ctypes.CDLL(_capi.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(_capi.EXPORTED) == names


def test_error_strings(pkg):
    for s in (0, -1, -2, -3, -4, -5, 1):
        assert pkg.hps_error_string(s).startswith("HPS_")


@pytest.mark.parametrize("dim,L,p", [(2, 0, 8), (2, 2, 8), (2, 1, 16), (3, 0, 6), (3, 1, 8), (3, 2, 6)])
def test_nodes_match_oracle_geometry(pkg, dim, L, p):
    from oracle import geometry as geo
    lo = (-1.0, -0.5, 0.25)[:dim]
    hi = tuple(x + 1.5 for x in lo)
    t = pkg.uniform_tree(dim, L, lo, hi)
    leaf, bdry = pkg.hps_nodes(t, p, p - 2)
    assert np.allclose(leaf, geo.leaf_nodes(dim, lo, hi, L, p), atol=1e-14)
    assert np.allclose(bdry, geo.root_boundary_points(dim, lo, hi, L, p - 2), atol=1e-14)


def test_invalid_arguments_are_rejected(pkg):
    t = pkg.uniform_tree(2, 2)
    with pytest.raises(pkg.HPSError) as e:
        pkg.hps_sizes(t, 8, 5)          # q != p - 2
    assert e.value.status == -1
    t.n_leaves = 7
    with pytest.raises(pkg.HPSError):
        pkg.hps_sizes(t, 8, 6)
    t = pkg.uniform_tree(2, 1, (0, 0), (1, 2))   # leaves must be squares
    with pytest.raises(pkg.HPSError):
        pkg.hps_nodes(t, 8, 6)
    t = pkg.uniform_tree(3, 1)
    # ItI is 2D only: rejected before any device work
    with pytest.raises(pkg.HPSError) as e:
        pkg.hps_build(t, 8, 6, pkg.HPS_ITI, eta=1.0)
    assert e.value.status == -1


def test_sizes(pkg):
    assert pkg.hps_sizes(pkg.uniform_tree(2, 6), 16, 14) == (4096, 256, 4 * 14 * 64)
    assert pkg.hps_sizes(pkg.uniform_tree(3, 3), 8, 6) == (512, 512, 6 * 36 * 64)


def _two_one_tree():
    from oracle import adaptive as ad
    leaves = [(1, (i, j, k)) for i in range(2) for j in range(2) for k in range(2) if (i, j, k) != (0, 0, 0)]
    leaves += ad.children_of(1, (0, 0, 0))
    leaves.remove((2, (1, 1, 1)))
    leaves += ad.children_of(2, (1, 1, 1))
    return ad.sort_leaves(ad.balance(leaves))


@pytest.mark.parametrize("p", [6, 8])
def test_adaptive_nodes_match_oracle(pkg, p):
    from oracle import adaptive as ad
    leaves = _two_one_tree()
    lo, hi = (-1.0, -0.5, 0.0), (1.0, 1.5, 2.0)
    t = pkg.adaptive_tree(leaves, lo, hi)
    nl, ppl, nr = pkg.hps_sizes(t, p, p - 2)
    assert (nl, ppl) == (len(leaves), p ** 3)
    leaf, bdry = pkg.hps_nodes(t, p, p - 2)
    assert np.allclose(leaf, ad.all_leaf_nodes(leaves, lo, hi, p), atol=1e-14)
    assert np.allclose(bdry, ad.root_boundary_points(leaves, lo, hi, p - 2), atol=1e-14)


def test_adaptive_trees_are_validated(pkg):
    from oracle import adaptive as ad
    leaves = _two_one_tree()
    # out of order
    bad = list(reversed(leaves))
    with pytest.raises(pkg.HPSError):
        pkg.hps_sizes(pkg.adaptive_tree(bad), 6, 4)
    # a gap in the tiling
    with pytest.raises(pkg.HPSError):
        pkg.hps_sizes(pkg.adaptive_tree(leaves[1:]), 6, 4)
    # not 2:1 balanced: one level-1 cell refined twice next to a level-1 leaf
    unb = [(1, (i, j, k)) for i in range(2) for j in range(2) for k in range(2) if (i, j, k) != (0, 0, 0)]
    unb += [lf for lf in ad.children_of(1, (0, 0, 0)) if lf[1] != (1, 1, 1)]
    unb += ad.children_of(2, (1, 1, 1))
    unb = ad.sort_leaves(unb)
    with pytest.raises(pkg.HPSError):
        pkg.hps_sizes(pkg.adaptive_tree(unb), 6, 4)
    assert pkg.hps_sizes(pkg.adaptive_tree(ad.sort_leaves(ad.balance(unb))), 6, 4)[0] > len(unb)


def test_server_options_are_validated(pkg):
    for kw in ({"n_slots": 0 - 1}, {"n_streams": 65}, {"max_batch": 257}, {"hbm_budget": -1}):
        with pytest.raises(pkg.HPSError) as e:
            pkg.Server(**kw)
        assert e.value.status == -1


def test_server_without_a_device_fails_cleanly(pkg):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(pkg.HPSError) as e:
        pkg.Server()
    assert e.value.status == -4


def test_plan_bytes_grows_with_the_tree(pkg):
    b = [pkg.hps_plan_bytes(pkg.uniform_tree(2, L), 16, 14, pkg.HPS_ITI) for L in (2, 3, 4)]
    assert b[0] < b[1] < b[2]
    assert 3.5 < b[2] / b[1] < 4.5
    with pytest.raises(pkg.HPSError):
        pkg.hps_plan_bytes(pkg.uniform_tree(3, 1), 8, 6, pkg.HPS_ITI)


def test_gemm_arguments_are_validated_before_any_device_work(pkg):
    """hps_gemm rejects bad dtype, mode and sizes, and returns for empty
    products, without touching a device (these run on a host with no GPU)."""
    from paper_2503_17535_gb300 import _capi
    L = _capi.lib()
    ok, bad = pkg.HPS_OK, -1
    # dtype / mode
    assert L.hps_gemm(7, 0, 4, 4, 4, 1, 1.0, None, 4, 16, None, 4, 16, 0.0, None, 4, 16, None) == bad
    assert L.hps_gemm(pkg.HPS_F64, 2, 4, 4, 4, 1, 1.0, None, 4, 16, None, 4, 16, 0.0, None, 4, 16, None) == bad
    # negative sizes, missing pointers, too-small leading dimensions
    assert L.hps_gemm(pkg.HPS_F64, 0, -1, 4, 4, 1, 1.0, 8, 4, 16, 8, 4, 16, 0.0, 8, 4, 16, None) == bad
    assert L.hps_gemm(pkg.HPS_F64, 0, 4, 4, 4, 1, 1.0, None, 4, 16, 8, 4, 16, 0.0, 8, 4, 16, None) == bad
    assert L.hps_gemm(pkg.HPS_F64, 0, 4, 4, 4, 1, 1.0, 8, 3, 16, 8, 4, 16, 0.0, 8, 4, 16, None) == bad
    assert L.hps_gemm(pkg.HPS_C128, 1, 4, 4, 4, 1, 1.0, 8, 4, 16, 8, 2, 16, 0.0, 8, 4, 16, None) == bad
    # empty products are no-ops
    assert L.hps_gemm(pkg.HPS_F64, 0, 0, 4, 4, 1, 1.0, 8, 1, 0, 8, 4, 16, 0.0, 8, 1, 0, None) == ok
    assert L.hps_gemm(pkg.HPS_F64, 0, 4, 4, 4, 0, 1.0, 8, 4, 16, 8, 4, 16, 0.0, 8, 4, 16, None) == ok


def test_fault_injection_hook_is_host_only(pkg):
    """Arming and disarming the allocation-failure hook and reading the
    allocation counter need no device."""
    n = pkg.hps_debug_alloc_count()
    pkg.hps_debug_fail_alloc(3)
    pkg.hps_debug_fail_alloc(0)
    pkg.hps_debug_fail_alloc(-5)
    assert pkg.hps_debug_alloc_count() == n


def test_debug_wait_timeout_rejects_bad_arguments(pkg):
    """Argument checks of hps_debug_wait_timeout happen on the host, before
    any device call."""
    from paper_2503_17535_gb300 import _capi
    assert pkg.hps_debug_wait_timeout(3, False, 1000, 0) == _capi.HPS_ERR_INVALID
    assert pkg.hps_debug_wait_timeout(-1, False, 1000, 0) == _capi.HPS_ERR_INVALID
    assert pkg.hps_debug_wait_timeout(0, False, 0, 0) == _capi.HPS_ERR_INVALID
    assert pkg.hps_debug_wait_timeout(0, False, (1 << 24) + 1, 0) == _capi.HPS_ERR_INVALID


def test_tuning_table_round_trip(pkg, tmp_path):
    """The batched LU's shape choices: compiled-in defaults equal the tuned
    table, values can be set and read back, bad parameters are refused; the
    autotuner's header writer emits every parameter."""
    import re as _re
    from paper_2503_17535_gb300 import _capi, autotune
    hdr = open(os.path.join(os.path.dirname(_capi.LIB_PATH), "csrc", "tuned.h")).read()
    table = {m: int(v) for m, v in _re.findall(r"#define (HPS_TUNED_\w+) (\d+)", hdr)}
    for name, macro in autotune.MACROS.items():
        assert pkg.hps_tune_get(name) == table[macro]
    old = pkg.hps_tune_get("lu_base_panels_few")
    pkg.hps_tune_set("lu_base_panels_few", 7)
    assert pkg.hps_tune_get("lu_base_panels_few") == 7
    pkg.hps_tune_set("lu_base_panels_few", old)
    lib = _capi.lib()
    assert lib.hps_tune_set(99, 1) == _capi.HPS_ERR_INVALID
    assert lib.hps_tune_set(0, -1) == _capi.HPS_ERR_INVALID
    out = tmp_path / "tuned.h"
    autotune.write_header(str(out), {k: v[0] for k, v in autotune.CANDIDATES.items()}, {"w": 1.0})
    got = dict(_re.findall(r"#define (HPS_TUNED_\w+) (\d+)", out.read_text()))
    assert set(got) == set(autotune.MACROS.values())
