"""Pins of the synthetic inputs: published SplitMix64 outputs, closed-form element matrices,
the de Rham property A^s G = 0 (Section 2, Eq. deRham) and the DoF counts of the meshes."""
import numpy as np
import pytest

import workloads as W
from workloads.rng import splitmix64


def test_splitmix64_published_sequence():
    # a SplitMix64 generator seeded with 0 first returns 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4
    g = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        out = splitmix64(np.array([0, g], dtype=np.uint64))
    assert int(out[0]) == 0xE220A8397B1DCDAF
    assert int(out[1]) == 0x6E789E6AA1B965F4


def test_uniform_streams_independent_and_in_range():
    a = W.uniform("rhs", 0, 1000)
    b = W.uniform("alpha", 0, 1000)
    assert a.min() >= -1 and a.max() < 1
    assert not np.allclose(a, b)
    # element i regenerates alone
    assert W.uniform("rhs", 0, 1, offset=537)[0] == a[537]
    assert abs(a.mean()) < 0.1


def test_hex_reference_element_closed_forms():
    K, M = W.hex_element_matrices()
    # x-edge (y,z) = (0,0): phi = (1-y)(1-z) e_x, curl = (0, -(1-y), (1-z)), |curl|^2 integrates to 2/3
    assert K[0, 0] == pytest.approx(2.0 / 3.0, rel=1e-14)
    # bilinear mass on the unit square for parallel edges: same 1/9, adjacent 1/18, opposite 1/36
    np.testing.assert_allclose(M[0, :4], [1 / 9, 1 / 18, 1 / 18, 1 / 36], rtol=1e-14)
    # edges of different directions are L2-orthogonal
    assert np.abs(M[:4, 4:]).max() == 0.0
    np.testing.assert_allclose(K, K.T, atol=1e-15)
    # K annihilates the local gradient of each vertex hat (local de Rham)
    verts = [(a, b, c) for c in (0, 1) for b in (0, 1) for a in (0, 1)]
    from workloads.meshes import HEX_LOCAL_EDGES
    for v in verts:
        g = np.zeros(12)
        for l, (d, off) in enumerate(HEX_LOCAL_EDGES):
            head = list(off)
            head[d] += 1
            g[l] = (tuple(head) == v) - (tuple(off) == v)
        assert np.abs(K @ g).max() < 1e-14


@pytest.mark.parametrize("n", [2, 3, 6])
def test_hex_counts_symmetry_de_rham(n):
    p = W.hex_problem(n, W.fields.log_uniform(n, 7), 0.3, with_parts=True)
    assert p["ndof"] == 3 * n * (n - 1) ** 2
    assert p["G"].shape == (p["ndof"], (n - 1) ** 3)
    A, As, G = p["A"], p["As"], p["G"]
    assert abs(A - A.T).max() <= 1e-14 * abs(A).max()
    assert abs(As @ G).max() <= 64 * np.finfo(float).eps * abs(As).max() * 8
    rows = np.diff(G.indptr)
    assert set(rows.tolist()) <= {1, 2}
    assert np.all(np.abs(G.data) == 1)
    assert np.diff(A.indptr).max() <= 33
    # SPD
    if p["ndof"] < 500:
        assert np.linalg.eigvalsh(A.toarray()).min() > 0


@pytest.mark.parametrize("N", [4, 16])
def test_triangle_counts_match_paper_sizes(N):
    # Tables 1-2 list n = 736 at L = 4 (N = 16): n = 3 N^2 - 2 N interior edges
    p = W.tri_problem(N, 1.0, 0.01, with_parts=True)
    assert p["ndof"] == 3 * N * N - 2 * N
    assert abs(p["As"] @ p["G"]).max() <= 1e-13 * abs(p["As"]).max()
    assert abs(p["A"] - p["A"].T).max() == 0.0


def test_quad_de_rham():
    p = W.quad_problem(8, W.fields.log_uniform(8, 1)[:64], 0.01, with_parts=True)
    assert abs(p["As"] @ p["G"]).max() <= 1e-13 * abs(p["As"]).max()


def test_checkerboard_blocks():
    a = W.fields.checkerboard(16, 8)
    assert set(np.unique(a)) == {1.0, 1e4}
    assert a[0] == 1.0 and a[2] == 1e4          # blocks of 2 elements along x
