"""Pins of the faceting oracle (Section 2.4.2): the faceted wavelet transform is
exactly the global one; the db8 4-level halo lies in [15(2^d-2), 15(2^d-1)];
apodisation weights are positive and sum to one per pixel."""
import math

import numpy as np
import pytest

from oracle import facets as fc
from oracle import wavelets as wv


@pytest.mark.parametrize("n1,n2,Qy,Qx", [(96, 96, 3, 3), (64, 80, 2, 3)])
def test_faceted_sara_equals_global(n1, n2, Qy, Qx):
    rng = np.random.default_rng(n1 + Qx)
    x = rng.standard_normal((2, n1, n2))
    c = wv.sara_analysis(x)
    w = rng.standard_normal(c.shape)
    got = np.full_like(c, np.nan)
    count = np.zeros(c.shape[-1], dtype=int)
    syn = np.zeros_like(x)
    for qy in range(Qy):
        for qx in range(Qx):
            idx, cq = fc.sara_facet_analysis(x, Qy, Qx, qy, qx)
            got[..., idx] = cq
            count[idx] += 1
            syn += fc.sara_facet_synthesis(w[..., idx], idx, n1, n2, Qy, Qx, qy, qx)
    assert np.all(count == 1)                       # ownership partitions the coefficients
    assert np.max(np.abs(got - c)) <= 1e-13 * np.max(np.abs(c))
    ref = wv.sara_synthesis(w, n1, n2)
    assert np.max(np.abs(syn - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_db8_halo_range_matches_paper():
    d, F = 4, 16
    halos = set()
    for a0 in range(512, 512 + 2 ** d):
        aJ = a0
        for _ in range(d):
            aJ = -((1 - aJ) // 2)
        halos.add(a0 - fc.sara_halo_start(aJ, F, d))
    assert min(halos) == 15 * (2 ** d - 2) and max(halos) == 15 * (2 ** d - 1)


def test_halo_is_minimal():
    # the owned coefficients of an interior facet depend on pixel column s0 (first halo
    # column) but not on column s0 - 1: an impulse there gives an exactly-zero response
    n, Q = 512, 2
    (s0, b0) = fc.sara_facet_input_1d(n, Q)[1]
    idx = fc.sara_owned_index(n, n, 1, Q, 0, 1)
    assert 256 - s0 == 210
    inside = np.zeros((1, n, n))
    inside[0, 200:260, s0] = 1.0
    outside = np.zeros((1, n, n))
    outside[0, 200:260, s0 - 1] = 1.0
    assert np.max(np.abs(wv.sara_analysis(inside)[..., idx])) > 0.0
    assert np.max(np.abs(wv.sara_analysis(outside)[..., idx])) == 0.0


@pytest.mark.parametrize("kind", ["triangular", "sine"])
@pytest.mark.parametrize("n,Q,rho", [(256, 4, 0.1), (100, 3, 0.25), (64, 1, 0.1), (1024, 8, 0.1)])
def test_nuclear_windows_partition_of_unity(kind, n, Q, rho):
    facets = fc.nuclear_facets(n, n, Q, Q, rho, kind)
    total = np.zeros((n, n))
    for f in facets:
        (r0, r1), (c0, c1), D = f["rows"], f["cols"], f["D"]
        assert np.all(D > 0)
        total[r0:r1, c0:c1] += D
    assert np.allclose(total, 1.0, atol=1e-14)
    tb = fc.tile_bounds(n, Q)
    for qy in range(Q):
        r0, r1 = facets[qy * Q]["rows"]
        o = 0 if qy == 0 else math.floor(rho * (tb[qy + 1] - tb[qy]))
        assert (r0, r1) == (tb[qy] - o, tb[qy + 1])


def test_triangular_window_values():
    (_, _, w), (_, _, w2) = fc.nuclear_facets_1d(20, 2, 0.3, "triangular")
    # overlap o = 3: later facet ramps 1/4, 2/4, 3/4; earlier facet 3/4, 2/4, 1/4
    assert np.allclose(w2[:3], [0.25, 0.5, 0.75])
    assert np.allclose(w[-3:], [0.75, 0.5, 0.25])


def test_step_size_condition():
    # tau (zeta ||D S~||^2 + kappa ||Psi^+||^2 + max_l eta_l ||Phi_l||^2) < 1 with
    # tau = 0.33, zeta = kappa = 1, eta_l = 1/||Phi_l||^2 (Section 3.2);
    # ||D S~||^2 = max over pixels of sum_q D_q^2 (block-diagonal operator)
    for kind in ("triangular", "sine"):
        n, Q = 256, 4
        s2 = np.zeros((n, n))
        for f in fc.nuclear_facets(n, n, Q, Q, 0.1, kind):
            (r0, r1), (c0, c1), D = f["rows"], f["cols"], f["D"]
            s2[r0:r1, c0:c1] += D * D
        assert 0.33 * (s2.max() + 1.0 + 1.0) < 1.0


@pytest.mark.parametrize("n1,n2,Qy,Qx", [(96, 96, 3, 3), (64, 80, 2, 3), (600, 600, 2, 2)])
def test_facet_local_analysis_equals_masked_global(n1, n2, Qy, Qx):
    """The crop-based facet analysis (for large images) gives exactly the owned
    coefficients of the transform of the masked full image, in the same order."""
    rng = np.random.default_rng(n1 * Qy + n2)
    x = rng.standard_normal((2, n1, n2))
    for qy in range(Qy):
        for qx in range(Qx):
            idx, ref = fc.sara_facet_analysis(x, Qy, Qx, qy, qx)
            idx2, got = fc.sara_facet_analysis_local(x, Qy, Qx, qy, qx)
            assert np.array_equal(idx, idx2)
            assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
