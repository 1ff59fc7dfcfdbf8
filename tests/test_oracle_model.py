"""Pins for the oracle's model layer: Slater-Koster blocks, periodic H and S, clusters, rounding.

Each check ties the oracle to something other than itself: the textbook SK
table values for bonds along the axes, rotation covariance of the p block,
symmetry of H and S, an explicit 27-image enumeration for cluster membership,
a second (global) builder for the projected matrices, torch's BF16 conversion.
"""
import numpy as np
import pytest

from oracle import sk as osk
from oracle.rounding import round_bf16, round_fp32
from synth import SK_CARBON_LIKE, WORKLOADS, lattice_positions, workload_positions

V = (-4.0, 4.5, 5.5, -1.8)


def test_sk_block_along_axes():
    """Bond of length d0 along +x, -y, +z: the table reduces to sigma/pi values (scale 1)."""
    d0 = 1.54
    B = osk.sk_block(np.array([d0, 0, 0]), V, d0)
    expect = np.array([[-4.0, 4.5, 0, 0], [-4.5, 5.5, 0, 0], [0, 0, -1.8, 0], [0, 0, 0, -1.8]])
    np.testing.assert_allclose(B, expect, atol=1e-15)
    B = osk.sk_block(np.array([0, -d0, 0]), V, d0)
    expect = np.array([[-4.0, 0, -4.5, 0], [0, -1.8, 0, 0], [4.5, 0, 5.5, 0], [0, 0, 0, -1.8]])
    np.testing.assert_allclose(B, expect, atol=1e-15)
    B = osk.sk_block(np.array([0, 0, 2 * d0]), V, d0)
    s = np.exp(-2.0)
    expect = s * np.array([[-4.0, 0, 0, 4.5], [0, -1.8, 0, 0], [0, 0, -1.8, 0], [-4.5, 0, 0, 5.5]])
    np.testing.assert_allclose(B, expect, atol=1e-15)


def test_sk_block_rotation_covariance():
    """A rotation Q of the bond rotates the p-p block as Q B Q^T and the s-p row as Q b."""
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    D = np.eye(4)
    D[1:, 1:] = Q
    for _ in range(5):
        d = rng.normal(size=3)
        np.testing.assert_allclose(osk.sk_block(Q @ d, V, 1.54), D @ osk.sk_block(d, V, 1.54) @ D.T, atol=1e-13)


def test_sk_block_reverse_bond_is_transpose():
    d = np.array([0.3, -1.1, 0.9])
    np.testing.assert_allclose(osk.sk_block(-d, V, 1.54), osk.sk_block(d, V, 1.54).T, atol=1e-15)


def test_vectorised_blocks_match_scalar():
    rng = np.random.default_rng(1)
    d = rng.normal(size=(20, 3)) * 1.5
    Bv = osk.sk_blocks(d, V, 1.54)
    for k in range(20):
        np.testing.assert_allclose(Bv[k], osk.sk_block(d[k], V, 1.54), rtol=0, atol=1e-14)


def test_lattice_counts_and_nearest_neighbour():
    pos, box = lattice_positions("diamond", 3.567, 2, 0.0, 0.0, 0)
    assert pos.shape == (64, 3)
    d = osk.min_image(pos[1:] - pos[0], box)
    r = np.sqrt((d * d).sum(1))
    assert np.isclose(r.min(), 3.567 * np.sqrt(3) / 4)
    assert np.sum(np.isclose(r, r.min())) == 4          # tetrahedral coordination
    w = WORKLOADS["fcc32k"]
    pos, _ = workload_positions(w)
    assert 0.94 * 32000 < pos.shape[0] < 0.96 * 32000    # 5% vacancies


def _images_within(pos, box, a, R):
    """Explicit enumeration of the 27 periodic images (valid when R < L/2)."""
    out = set()
    for sx in (-1, 0, 1):
        for sy in (-1, 0, 1):
            for sz in (-1, 0, 1):
                d = pos + np.array([sx, sy, sz]) * box - pos[a]
                out |= set(np.nonzero((d * d).sum(1) <= R * R)[0].tolist())
    return np.array(sorted(out))


def test_cluster_membership_matches_image_enumeration():
    w = WORKLOADS["diamond512"]
    pos, box = workload_positions(w)
    for a in (0, 17, 300, 511):
        np.testing.assert_array_equal(osk.cluster_atoms(pos, box, a, w.R), _images_within(pos, box, a, w.R))


def test_global_matrices_symmetric_and_cluster_is_restriction():
    pos, box = lattice_positions("diamond", 3.567, 2, 0.1, 0.0, 7)
    g = osk.global_bsr(pos, box, SK_CARBON_LIKE)
    H = osk.bsr_to_dense(g["row_ptr"], g["col"], g["H"])
    S = osk.bsr_to_dense(g["row_ptr"], g["col"], g["S"])
    np.testing.assert_allclose(H, H.T, atol=1e-14)
    np.testing.assert_allclose(S, S.T, atol=1e-14)
    assert np.all(np.diag(S) == 1.0)
    for a in (0, 5, 63):
        cl = osk.cluster_atoms(pos, box, a, 3.0)
        Hc, Sc = osk.cluster_matrices(pos, box, cl, SK_CARBON_LIKE)
        orb = (4 * cl[:, None] + np.arange(4)).ravel()
        np.testing.assert_allclose(Hc, H[np.ix_(orb, orb)], atol=1e-14)
        np.testing.assert_allclose(Sc, S[np.ix_(orb, orb)], atol=1e-14)


def test_overlap_is_positive_definite_diamond512():
    """The 512-atom workload's S (M = 2048) admits a dense Cholesky factorisation."""
    w = WORKLOADS["diamond512"]
    pos, box = workload_positions(w)
    allat = np.arange(pos.shape[0])
    _, S = osk.cluster_matrices(pos, box, allat, w.sk)
    np.linalg.cholesky(S)
    lam = np.linalg.eigvalsh(S)
    assert 0.3 < lam[0] < 1.0


def test_bf16_rounding_matches_torch_and_ties_to_even():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.normal(size=2000) * 10.0 ** rng.integers(-6, 3, 2000),
                        [1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 2.0 ** -8), 0.0]])
    f32 = x.astype(np.float32)
    ref = torch.from_numpy(f32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(round_bf16(x), ref)
    assert round_bf16(np.array([1 + 2.0 ** -8]))[0] == 1.0                # tie -> even (down)
    assert round_bf16(np.array([1 + 3 * 2.0 ** -8]))[0] == 1 + 2.0 ** -6  # tie -> even (up)
    assert round_fp32(np.array([1 + 2.0 ** -30]))[0] == 1.0
