"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle (oracle/das_oracle.c) against something other than
itself: hand-computed geometry with exact distances, numpy's linear
interpolation, integer lattice counts, scipy's analytic-signal demodulation,
the exact conjugate-transpose identity, a dense matrix built column by column,
central finite differences, and the problem sizes the paper prints.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2606_13259_gb300 import synth as S

MM = 1e-3
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def one_voxel(p_mm, elems_mm, tx, f_number, K=1024, fs=30e6, c=1540.0, iq=False, fd=0.0,
              t0_offset=True):
    """A single-voxel scene.  tx: list of (kind, vec) with vec in mm for
    diverging sources and unitless for plane-wave directions."""
    pos = np.array(elems_mm, dtype=np.float64) * MM
    nrm = np.tile([0.0, 0.0, 1.0], (len(pos), 1))
    kinds = np.array([k for k, _ in tx], dtype=np.int32)
    vecs = np.array([np.array(v, float) * (MM if k == S.TX_DIVERGING else 1.0) for k, v in tx])
    return S.Scene("pin", 1, 1, 1, tuple(np.array(p_mm, float) * MM), (0.1 * MM,) * 3, pos, nrm, kinds,
                   vecs, t0_offset=t0_offset, c=c, fs=fs, f_demod=fd, f_number=f_number, K=K, iq=iq)


def rng_y(scene, B, seed):
    return S.random_channels(scene, B, seed).numpy()


# ---------------------------------------------------------------- delays + interpolation

# voxel (0, 0, 4) mm, element (3, 0, 0) mm: receive path 5 mm exactly.
# diverging source (0, 0, -3) mm: ||p - v|| = 7 mm, ||v - o|| = 3 mm.
# plane direction (0.6, 0, 0.8): d . p = 3.2 mm.
INTERP_CASES = [
    ("diverging", [(S.TX_DIVERGING, (0, 0, -3))], True, (7 - 3 + 5)),
    ("diverging_no_t0", [(S.TX_DIVERGING, (0, 0, -3))], False, (7 + 5)),
    ("plane", [(S.TX_PLANE, (0.6, 0.0, 0.8))], True, (3.2 + 5)),
    ("photoacoustic", [(S.TX_NONE, (0, 0, 0))], True, 5),
]


@pytest.mark.parametrize("name,tx,t0,path_mm", INTERP_CASES, ids=[c[0] for c in INTERP_CASES])
def test_single_term_is_numpy_interp(oracle, name, tx, t0, path_mm):
    """One voxel, one element, one transmit: Eq. 2 reduces to linear
    interpolation of the channel at tau*fs (numpy.interp), Sec. 2."""
    sc = one_voxel((0, 0, 4), [(3, 0, 0)], tx, f_number=0.5, t0_offset=t0)
    y = rng_y(sc, 1, 11)
    tau_s = path_mm * MM * sc.fs / sc.c
    expect = np.interp(tau_s, np.arange(sc.K), y[0, 0, 0])
    x = oracle.forward(sc, y)
    assert abs(x[0, 0].real - expect) <= 1e-12 * max(1.0, abs(expect))
    assert x[0, 0].imag == 0.0


def test_single_term_masked_outside_aperture(oracle):
    """f-number 1 at depth 4 mm admits lateral offsets up to 2 mm; the element
    is 3 mm off axis, so the sum is empty."""
    sc = one_voxel((0, 0, 4), [(3, 0, 0)], [(S.TX_DIVERGING, (0, 0, -3))], f_number=1.0)
    x = oracle.forward(sc, rng_y(sc, 1, 12))
    assert x[0, 0] == 0.0


@pytest.mark.parametrize("K,valid", [(177, True), (176, False), (175, False)])
def test_sample_range_edge(oracle, K, valid):
    """tau*fs = 270000/1540 = 175.32..., so k = 175: the term needs k <= K - 2."""
    sc = one_voxel((0, 0, 4), [(3, 0, 0)], [(S.TX_DIVERGING, (0, 0, -3))], f_number=0.5, K=K)
    y = rng_y(sc, 1, 13)
    x = oracle.forward(sc, y)
    if valid:
        expect = np.interp(270000 / 1540, np.arange(K), y[0, 0, 0])
        assert abs(x[0, 0].real - expect) <= 1e-12 * max(1.0, abs(expect))
    else:
        assert x[0, 0] == 0.0


def test_ramp_sums_delays_exactly(oracle):
    """Linear interpolation is exact on a ramp y[k] = k, so x = sum of w * tau*fs.
    Voxel (0, 0, 12) mm; four elements on a 5 mm ring (receive path 13 mm) and
    one at 7 mm (outside the f-number-1 aperture of half width 6 mm);
    sources (0, 0, -5) mm (transmit path 17 - 5 = 12 mm) and (9, 0, 0) mm
    (15 - 9 = 6 mm)."""
    ring = [(3, 4, 0), (-4, 3, 0), (5, 0, 0), (0, -5, 0)]
    sc = one_voxel((0, 0, 12), ring + [(7, 0, 0)],
                   [(S.TX_DIVERGING, (0, 0, -5)), (S.TX_DIVERGING, (9, 0, 0))], f_number=1.0, K=4096)
    y = np.broadcast_to(np.arange(sc.K, dtype=np.float32), (1, sc.Q, sc.M, sc.K)).copy()
    expect = 4 * ((12 + 13) + (6 + 13)) * MM * 30e6 / 1540
    x = oracle.forward(sc, y)
    assert abs(x[0, 0].real - expect) <= 1e-12 * expect


@pytest.mark.parametrize("f_number,inside", [(1.2, True), (1.2 * (1 + 1e-5), False)])
def test_aperture_tie_is_inside(oracle, f_number, inside):
    """At depth 12 mm and f-number 1.2 the aperture half width is exactly 5 mm,
    the radius of the element ring: exact ties count as inside (reading R6);
    an f-number 1e-5 larger leaves them outside."""
    ring = [(3, 4, 0), (-4, 3, 0), (5, 0, 0), (0, -5, 0)]
    sc = one_voxel((0, 0, 12), ring, [(S.TX_DIVERGING, (0, 0, -5))], f_number=f_number, K=4096)
    y = np.broadcast_to(np.arange(sc.K, dtype=np.float32), (1, sc.Q, sc.M, sc.K)).copy()
    x = oracle.forward(sc, y)
    expect = 4 * (12 + 13) * MM * 30e6 / 1540 if inside else 0.0
    assert abs(x[0, 0].real - expect) <= 1e-12 * max(expect, 1.0)


def test_iq_constant_gives_phasor_sum(oracle):
    """IQ data equal to 1 everywhere give x = sum w e^{+i 2 pi f_d tau}: with
    f_d / fs = 1/4 and the ring geometry above (paths 25 and 19 mm), the two
    phasors are at 2 pi * (25 mm, 19 mm) * fs / c / 4."""
    ring = [(3, 4, 0), (-4, 3, 0), (5, 0, 0), (0, -5, 0)]
    sc = one_voxel((0, 0, 12), ring, [(S.TX_DIVERGING, (0, 0, -5)), (S.TX_DIVERGING, (9, 0, 0))],
                   f_number=1.0, K=4096, iq=True, fd=7.5e6)
    y = np.ones((1, sc.Q, sc.M, sc.K), dtype=np.complex64)
    t1, t2 = 25 * MM * 30e6 / 1540, 19 * MM * 30e6 / 1540
    expect = 4 * (np.exp(2j * np.pi * t1 / 4) + np.exp(2j * np.pi * t2 / 4))
    x = oracle.forward(sc, y)
    assert abs(x[0, 0] - expect) <= 1e-12 * abs(expect) + 1e-12


# ---------------------------------------------------------------- aperture

def lattice_counts_small():
    """Elements inside the f-number-1 aperture of every voxel of the small
    scene, by exact integer arithmetic in units of 0.05 mm: elements at
    6 j - 45, voxels at 4 i - 62 laterally and 100 + 4 i in depth; the element
    is inside when 4 rho^2 <= z^2 (ties included)."""
    j = np.arange(16)
    ex, ey = np.meshgrid(6 * j - 45, 6 * j - 45, indexing="xy")
    ex, ey = ex.ravel().astype(np.int64), ey.ravel().astype(np.int64)
    i = np.arange(32)
    vz, vy, vx = np.meshgrid(100 + 4 * i, 4 * i - 62, 4 * i - 62, indexing="ij")
    vx, vy, vz = vx.ravel()[:, None], vy.ravel()[:, None], vz.ravel()[:, None]
    rho2 = (vx - ex[None]) ** 2 + (vy - ey[None]) ** 2
    inside = 4 * rho2 <= vz ** 2
    return inside.sum(1)


def test_constant_data_counts_aperture(oracle):
    """y = 1 (RF) makes every term's interpolated sample 1, so x_n is the number
    of elements in voxel n's aperture (all delays of this scene are in range)."""
    sc = S.scene_small()
    counts = lattice_counts_small()
    y = np.ones((1, sc.Q, sc.M, sc.K), dtype=np.float32)
    x = oracle.forward(sc, y)
    np.testing.assert_array_equal(x[0].real, counts.astype(np.float64))


def test_transmit_weight_multiplies(oracle):
    """A per-voxel transmit weight table [q][n] scales each transmit's terms."""
    sc = S.scene_small().with_(K=512)
    sc = sc.with_(tx_kind=np.array([0, 0], np.int32), tx_vec=np.array([[0, 0, -10 * MM], [1 * MM, 0, -10 * MM]]))
    rng = np.random.default_rng(3)
    wtx = rng.random((2, sc.N)).astype(np.float32)
    counts = lattice_counts_small()
    y = np.ones((1, sc.Q, sc.M, sc.K), dtype=np.float32)
    x = oracle.forward(sc.with_(w_tx=wtx), y)
    expect = (wtx.astype(np.float64).sum(0)) * counts
    np.testing.assert_allclose(x[0].real, expect, rtol=1e-12)


def test_small_scene_has_no_near_ties(oracle):
    """No voxel-element pair of the small scene sits near the aperture edge
    without sitting exactly on it, so float32 and float64 decide alike."""
    assert oracle.count_near_ties(S.scene_small(), 1e-5) == 0


def test_count_active_small_scene_is_lattice_count(oracle):
    """Every delay of the small scene lies in range (K = 512; with K = 4096 also
    for a second, laterally shifted source), so the number of contributing
    terms is Q times the exact integer count of aperture elements summed over
    the voxels (Eq. 2 with the range rule of the text after it)."""
    sc = S.scene_small()
    per_tx = int(lattice_counts_small().sum())
    assert oracle.count_active(sc) == per_tx
    two = sc.with_(K=4096, tx_kind=np.array([0, 0], np.int32),
                   tx_vec=np.array([[0.0, 0.0, -10 * MM], [1.0 * MM, 0.0, -10 * MM]]))
    assert oracle.count_active(two) == 2 * per_tx


@pytest.mark.parametrize("K,count", [(489, 8), (488, 4), (372, 4), (371, 0)])
def test_count_active_range_edges(oracle, K, count):
    """Ring scene: voxel (0, 0, 12) mm, four elements on a 5 mm ring (receive
    path 13 mm) inside the f-number-1 aperture and one at 7 mm outside it;
    source (0, 0, -5) mm gives the path 12 + 13 = 25 mm, i.e. tau fs =
    750000 / 1540 = 487.01 (k = 487), source (9, 0, 0) mm gives 6 + 13 = 19 mm,
    i.e. 570000 / 1540 = 370.13 (k = 370).  A term counts when k <= K - 2."""
    ring = [(3, 4, 0), (-4, 3, 0), (5, 0, 0), (0, -5, 0)]
    sc = one_voxel((0, 0, 12), ring + [(7, 0, 0)],
                   [(S.TX_DIVERGING, (0, 0, -5)), (S.TX_DIVERGING, (9, 0, 0))], f_number=1.0, K=K)
    assert oracle.count_active(sc) == count


def test_count_near_ties_hand_built(oracle):
    """Voxel (0, 0, 12) mm at f-number 1.2: the aperture half width is exactly
    5 mm.  The four ring elements sit exactly on it (ties, never counted), one
    element is 1e-7 off in rho^2 (5 (1 + 5e-8) mm), one about 4e-5 off
    (5.0001 mm) and one far inside (3 mm, rho^2 off by 0.64)."""
    ring = [(3, 4, 0), (-4, 3, 0), (5, 0, 0), (0, -5, 0)]
    near = [(5 * (1 + 5e-8), 0, 0), (-5.0001, 0, 0), (0, 3, 0)]
    sc = one_voxel((0, 0, 12), ring + near, [(S.TX_DIVERGING, (0, 0, -5))], f_number=1.2)
    assert oracle.count_near_ties(sc, 1e-5) == 1
    assert oracle.count_near_ties(sc, 1e-4) == 2
    assert oracle.count_near_ties(sc, 1.0) == 3
    assert oracle.count_near_ties(one_voxel((0, 0, 12), ring, [(S.TX_DIVERGING, (0, 0, -5))],
                                            f_number=1.2), 1.0) == 0
    assert oracle.count_near_ties(sc.with_(f_number=0.0), 1.0) == 0


# ---------------------------------------------------------------- point reflectors

def test_point_reflectors_peak_at_their_voxels(oracle):
    """Reflectors simulated at voxel centres (acquisition model in synth.py)
    beamform to a local maximum at exactly those voxels (RF)."""
    sc = S.scene_small()
    pos, amp = S.phantom(sc, 0, S.SMALL_POINTS, seed=1)
    y = S.simulate(sc, pos, amp).numpy()[None]
    img = oracle.forward(sc, y)[0].real.reshape(sc.nz, sc.ny, sc.nx)
    for ix, iy, iz in S.SMALL_POINTS:
        sub = img[iz - 3:iz + 4, iy - 3:iy + 4, ix - 3:ix + 4]
        assert np.unravel_index(np.argmax(sub), sub.shape) == (3, 3, 3)


def test_iq_phase_matches_analytic_signal(oracle):
    """Reading R5 against textbook demodulation: take RF echoes of the point
    reflectors, form the analytic signal with scipy.signal.hilbert and
    demodulate it (IQ[k] = a[k] e^{-i 2 pi f_d k / fs}).  Beamforming the IQ data
    with the e^{+i 2 pi f_d tau} factor must match beamforming the analytic
    signal itself (f_d = 0) in phase at each reflector, and be at least as
    coherent (linear interpolation of the carrier-rate analytic signal loses
    some amplitude; of the baseband signal, less).  With the opposite sign the
    IQ terms would not add in phase and the sum would collapse."""
    from scipy.signal import hilbert

    sc = S.scene_small()
    pos, amp = S.phantom(sc, 0, S.SMALL_POINTS, seed=1)
    rf = S.simulate(sc, pos, amp).numpy().astype(np.float64)
    analytic = hilbert(rf, axis=-1)
    k = np.arange(sc.K)
    iq = analytic * np.exp(-2j * np.pi * 7.5e6 * k / sc.fs)
    x_iq = oracle.forward(sc.with_(iq=True, f_demod=7.5e6), iq.astype(np.complex64)[None])[0]
    x_an = oracle.forward(sc.with_(iq=True, f_demod=0.0), analytic.astype(np.complex64)[None])[0]
    for ix, iy, iz in S.SMALL_POINTS:
        n = sc.voxel_index(ix, iy, iz)
        assert 0.95 < abs(x_iq[n]) / abs(x_an[n]) < 1.5
        assert abs(np.angle(x_iq[n] / x_an[n])) < 0.1
        assert abs(np.angle(x_iq[n])) < 0.1


# ---------------------------------------------------------------- linearity and the adjoint

def test_linearity(oracle):
    sc = S.scene_tiny(iq=True, n=(4, 3, 5), elems=(3, 2), n_tx=3, f_number=1.0)
    rng = np.random.default_rng(5)
    y1 = rng.standard_normal((2, sc.Q, sc.M, sc.K)) + 1j * rng.standard_normal((2, sc.Q, sc.M, sc.K))
    y2 = rng.standard_normal((2, sc.Q, sc.M, sc.K)) + 1j * rng.standard_normal((2, sc.Q, sc.M, sc.K))
    a, b = 0.7 - 1.3j, -2.1 + 0.4j
    lhs = oracle.forward_f64(sc, a * y1 + b * y2)
    rhs = a * oracle.forward_f64(sc, y1) + b * oracle.forward_f64(sc, y2)
    assert np.abs(lhs - rhs).max() <= 1e-13 * np.abs(rhs).max()


ADJ_SCENES = {
    "tiny_iq_full_aperture": lambda: S.scene_tiny(iq=True, n=(3, 3, 3), elems=(2, 2), n_tx=2, f_number=0.0),
    "tiny_rf_masked": lambda: S.scene_tiny(iq=False, n=(5, 4, 3), elems=(3, 3), n_tx=2, f_number=1.0),
    "small_iq": lambda: S.scene_small_iq(),
    "mixed_transmits_out_of_range": lambda: S.scene_tiny(iq=True, n=(6, 5, 4), elems=(4, 3), n_tx=3,
                                                         f_number=0.8, K=48).with_(
        tx_kind=np.array([S.TX_DIVERGING, S.TX_PLANE, S.TX_NONE], np.int32),
        tx_vec=np.array([[0.2 * MM, 0.1 * MM, -4 * MM], [0.3, 0.0, math.sqrt(1 - 0.09)], [0, 0, 0]])),
}


@pytest.mark.parametrize("name", list(ADJ_SCENES))
def test_adjoint_dot_product(oracle, name):
    """<A y, x> = <y, A^H x> to 1e-12 relative on seeded complex data."""
    sc = ADJ_SCENES[name]()
    rng = np.random.default_rng(7)
    B = 2
    y = rng.standard_normal((B, sc.Q, sc.M, sc.K)) + (1j * rng.standard_normal((B, sc.Q, sc.M, sc.K)) if sc.iq else 0)
    x = rng.standard_normal((B, sc.N)) + 1j * rng.standard_normal((B, sc.N))
    Ay = oracle.forward_f64(sc, y)
    AHx = oracle.adjoint(sc, x).reshape(y.shape)
    lhs = np.vdot(Ay, x)
    rhs = np.vdot(y, AHx)
    scale = np.linalg.norm(Ay) * np.linalg.norm(x)
    assert abs(lhs - rhs) <= 1e-12 * scale
    if not sc.iq:
        # real data: only the real part of y is seen by the forward map
        assert np.vdot(y.real, AHx.real) == pytest.approx(lhs.real, rel=1e-12, abs=1e-12 * scale)


def test_adjoint_equals_dense_conjugate_transpose(oracle):
    """Brute force on a tiny problem: build A column by column from the forward
    map applied to unit channel vectors, then A^H x must equal the adjoint."""
    sc = S.scene_tiny(iq=True, n=(3, 2, 2), elems=(2, 2), n_tx=2, f_number=1.0, K=48)
    D = sc.Q * sc.M * sc.K
    eye = np.eye(D).reshape(D, sc.Q, sc.M, sc.K)
    A = oracle.forward_f64(sc, eye).T                      # (N, D): column j = A e_j
    Ai = oracle.forward_f64(sc, 1j * eye).T
    np.testing.assert_allclose(Ai, 1j * A, atol=1e-14)     # complex-linear
    rng = np.random.default_rng(9)
    x = rng.standard_normal((1, sc.N)) + 1j * rng.standard_normal((1, sc.N))
    adj = oracle.adjoint(sc, x).reshape(-1)
    np.testing.assert_allclose(adj, A.conj().T @ x[0], rtol=0, atol=1e-13 * np.abs(adj).max())
    rows = [3, 0, 5]
    sub = oracle.adjoint(sc, x, rows=rows)
    np.testing.assert_array_equal(sub[0], adj.reshape(sc.Q * sc.M, sc.K)[rows])


def test_voxel_subset_matches_full(oracle):
    sc = S.scene_small_iq()
    y = rng_y(sc, 2, 21)
    full = oracle.forward(sc, y)
    vox = [0, 5, 12345, sc.N - 1, 777]
    np.testing.assert_array_equal(oracle.forward(sc, y, voxels=vox), full[:, vox])


# ---------------------------------------------------------------- sound-speed gradient

def diff_scene_small(c):
    """The small geometry with IQ data and a lateral 2-source lattice."""
    return S.scene_small_iq().with_(c=c, tx_kind=np.array([0, 0], np.int32),
                                    tx_vec=np.array([[-1.5 * MM, 0, -10 * MM], [1.5 * MM, 0, -10 * MM]]))


def _loss(oracle, sc, y, c):
    x = oracle.forward(sc.with_(c=c), y)
    return oracle.loss_and_cotangent(x)


@pytest.mark.parametrize("c_true,offset", [(1540.0, -40.0), (1540.0, 40.0), (1500.0, 40.0)])
def test_grad_c_matches_central_differences(oracle, c_true, offset):
    """dL/dc for L = -sum|x|^4 / (sum|x|^2)^2 against central differences, and
    sign(dL/dc) = sign(c_bf - c_true).  With h = 0.05 m/s a delay moves by about
    0.01 sample, so a few percent of the terms cross an interpolation kink and
    the difference quotient is good to a few 1e-3; with h = 1e-4 m/s it agrees
    to 1e-4."""
    sc = diff_scene_small(c_true)
    pos, amp = S.phantom(sc, 400, S.SMALL_POINTS, seed=5)
    y = S.simulate(sc, pos, amp).numpy()[None]
    c_bf = c_true + offset
    L, g = _loss(oracle, sc, y, c_bf)
    dLdc = oracle.grad_c(sc.with_(c=c_bf), y, g)
    for h, tol in [(0.05, 5e-3), (1e-4, 1e-4)]:
        fd = (_loss(oracle, sc, y, c_bf + h)[0] - _loss(oracle, sc, y, c_bf - h)[0]) / (2 * h)
        assert abs(dLdc - fd) <= tol * abs(fd)
    assert np.sign(dLdc) == np.sign(offset)


def test_grad_c_linear_functional_fd(oracle):
    """Re sum conj(g) dx/dc for a fixed random g against central differences of
    Re sum conj(g) x(c) on a voxel subset (the functional is linear in x).
    White-noise data make every interpolation kink count, so the step is small
    enough (1e-5 m/s, about 3e-6 sample) that almost no term crosses one."""
    sc = diff_scene_small(1540.0)
    y = rng_y(sc, 1, 31)
    vox = np.arange(0, sc.N, 97)
    rng = np.random.default_rng(4)
    g = rng.standard_normal((1, vox.size)) + 1j * rng.standard_normal((1, vox.size))
    an = oracle.grad_c(sc, y, g, voxels=vox)
    h = 1e-5
    f = lambda c: np.real(np.vdot(g, oracle.forward(sc.with_(c=c), y, voxels=vox)))
    fd = (f(1540.0 + h) - f(1540.0 - h)) / (2 * h)
    assert abs(an - fd) <= 1e-6 * abs(fd)


# ---------------------------------------------------------------- paper's printed sizes

def test_paper_problem_sizes():
    """Sec. 2: N = 128^3, M = 32^2, Q = 16 give about 3.4e10 accumulations per
    volume, and a float32 delay table of about 1.37e11 bytes (128 GiB)."""
    g = json.load(open(os.path.join(GOLDEN, "paper_sizes.json")))
    sc = S.scene_paper()
    assert (sc.N, sc.M, sc.Q) == (g["N"], g["M"], g["Q"])
    terms = sc.N * sc.M * sc.Q
    assert terms == pytest.approx(g["accumulations_per_volume_approx"], rel=0.02)
    assert 4 * terms == pytest.approx(g["delay_table_bytes_approx"], rel=0.01)
    assert 4 * terms / 2 ** 30 == pytest.approx(g["delay_table_gib_approx"], rel=0.01)
