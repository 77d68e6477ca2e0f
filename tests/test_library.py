"""CPU-side checks of the C ABI library: it builds for sm_103a, loads, and
exports every entry point include/knng.h declares; host-only entry points
answer without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1701_08475_gb300 import build
    build.build()
    import paper_1701_08475_gb300 as knng
    return knng.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "knng.h")).read()
    return sorted(set(re.findall(r"KNNG_API\s+[\w\s\*]*?\b(knng_\w+)\s*\(", text)))


def test_header_declares_the_abi():
    names = _declared()
    for want in ("knng_build", "knng_build_ex", "knng_refine", "knng_partition", "knng_leaf_update",
                 "knng_exact", "knng_recall", "knng_last_error", "knng_workspace_bytes"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_1701_08475_gb300", "libknng.so")],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (knng_\w+)", out))
    assert set(_declared()) <= exported
    # nothing but the C ABI is exported
    assert exported == set(_declared())
    for name in _declared():
        assert getattr(lib, name) is not None


def test_library_is_built_for_sm103a(lib):
    out = subprocess.run(["cuobjdump", "--list-elf", os.path.join(ROOT, "paper_1701_08475_gb300", "libknng.so")],
                         capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def test_host_only_entry_points(lib):
    import paper_1701_08475_gb300 as knng
    p = knng.default_params()
    assert (p.k, p.leaf_max, p.tree_passes, p.refine_rounds, p.twomeans_iters) == (10, 64, 1, 0, 4)
    assert knng.knng_tree_depth(1_000_000, 128) == 13
    assert knng.knng_tree_depth(10_000, 64) == 8
    assert knng.knng_tree_depth(50, 64) == 0
    assert knng.knng_tree_depth(0, 64) == -1
    p2 = knng.default_params(k=20, leaf_max=128, tree_passes=3, refine_rounds=4)
    ws = knng.knng_workspace_bytes(1_000_000, 128, p2)
    # graph double buffer + reverse lists at least; bounded offer budget
    assert 4 * 1_000_000 * 20 * 8 <= ws < 16 << 30
    bad = knng.default_params(k=20, leaf_max=30)   # leaf_max < 2(k+1)
    assert knng.knng_workspace_bytes(1000, 8, bad) == 0
    assert b"leaf_max" in lib.knng_last_error()


def test_invalid_arguments_are_rejected_without_a_gpu(lib):
    import numpy as np
    import paper_1701_08475_gb300 as knng
    X = np.zeros((10, 4), np.float32)
    with pytest.raises(knng.KnngError) as e:
        knng.knng_build(X, k=10, leaf_max=64)      # n <= k
    assert e.value.code == -1
    with pytest.raises(knng.KnngError):
        knng.knng_build(X, k=3, leaf_max=7)        # leaf_max < 2(k+1)
    with pytest.raises(knng.KnngError):
        knng.knng_build_ex(X, knng.default_params(k=3, leaf_max=64, precision=7))


def test_rvq_arguments_are_rejected_without_a_gpu(lib):
    import numpy as np
    import paper_1701_08475_gb300 as knng
    assert {"knng_rvq_train", "knng_rvq_index", "knng_rvq_seeds", "knng_search"} <= set(_declared())
    X = np.zeros((10, 4), np.float32)
    for W1, W2 in ((0, 4), (300, 4), (11, 4), (4, 257)):
        with pytest.raises(knng.KnngError) as e:
            knng.knng_rvq_train(X, W1=W1, W2=W2)
        assert e.value.code == -1
    with pytest.raises(knng.KnngError):
        knng.knng_rvq_train(X, W1=4, W2=4, iters=-1)
    w = np.zeros((4, 4), np.float32)
    off = np.zeros(17, np.int32)
    ids = np.zeros(0, np.int32)
    with pytest.raises(knng.KnngError):
        knng.knng_rvq_seeds(w, w, off, ids, X, 5, 3)          # probe1 > W1
    with pytest.raises(knng.KnngError):
        knng.knng_rvq_seeds(w, w, off, ids, X, 0, 3)          # probe1 < 1
    big = np.zeros((256, 4), np.float32)
    with pytest.raises(knng.KnngError):
        knng.knng_rvq_seeds(big, big, np.zeros(65537, np.int32), ids, X, 33, 3)   # 33 * 256 keys > 8192


def test_sampled_join_parameters_without_a_gpu(lib):
    import numpy as np
    import paper_1701_08475_gb300 as knng
    p = knng.default_params()
    assert p.sample == 0 and knng.KNNG_JOIN_SAMPLED == 2
    X = np.zeros((500, 4), np.float32)
    for sample in (0, 5, -1):                           # outside [1, k / 2] for k = 8
        q = knng.default_params(k=8, leaf_max=64, refine_rounds=1, join_mode=knng.KNNG_JOIN_SAMPLED, sample=sample)
        with pytest.raises(knng.KnngError) as e:
            knng.knng_build_ex(X, q)
        assert e.value.code == -1
    q = knng.default_params(k=8, leaf_max=64, refine_rounds=1, join_mode=3)
    with pytest.raises(knng.KnngError):
        knng.knng_build_ex(X, q)
