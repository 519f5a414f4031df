"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test ties one function of the oracle to a closed form, a dense
brute-force computation in real space, an invariant, or a textbook routine,
chosen so that a plausible slip (a swapped axis, a dropped factor, a wrong
sign or index) fails at least one of them. tests/test_oracle_planted.py
plants such slips and checks that they are caught.
"""
import numpy as np
import pytest
import scipy.linalg

import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _cn_dense(Op, psi, T, S):
    """S Crank-Nicolson steps with the dense real-space operator."""
    n = Op.shape[0]
    I = np.eye(n)
    dt = T / S
    step = np.linalg.solve(I - 0.5 * dt * Op, I + 0.5 * dt * Op)
    for _ in range(S):
        psi = step @ psi
    return psi


def _expm_sym(Op, psi, T):
    w, V = np.linalg.eigh(Op)
    return V @ (np.exp(T * w) * (V.T @ psi))


# --------------------------------------------------------------------------
# transforms and symbols
# --------------------------------------------------------------------------

@pytest.mark.parametrize("H,W", [(6, 10), (8, 4), (5, 7)])
def test_central_difference_symbol(oracle_mod, H, W):
    """Theorem 2: the DFT maps the periodic central difference along x to
    multiplication by i sin(2 pi l/W), along y by i sin(2 pi k/H)."""
    rng = np.random.default_rng(7)
    psi = rng.standard_normal((H, W))
    dx = 0.5 * (np.roll(psi, -1, axis=1) - np.roll(psi, 1, axis=1))
    dy = 0.5 * (np.roll(psi, -1, axis=0) - np.roll(psi, 1, axis=0))
    wx, wy = oracle_mod.omegas(H, W)
    P = np.fft.fft2(psi)
    np.testing.assert_allclose(np.fft.fft2(dx), 1j * wx[None, :] * P, atol=1e-12)
    np.testing.assert_allclose(np.fft.fft2(dy), 1j * wy[:, None] * P, atol=1e-12)


def test_forward_inverse_roundtrip(oracle_mod):
    v = synth.random_volume(3, 6, 10, 1)
    np.testing.assert_allclose(oracle_mod.inverse(oracle_mod.forward(v)), v, atol=1e-14)
    # unnormalised forward: the zero frequency is the plain sum of each plane
    np.testing.assert_allclose(oracle_mod.forward(v)[:, 0, 0], v.sum(axis=(1, 2)), atol=1e-12)


# --------------------------------------------------------------------------
# Theorem 2: the Fourier path integrates the real-space operator exactly
# --------------------------------------------------------------------------

@pytest.mark.parametrize("H,W,N,conv", [(4, 6, 4, 0), (6, 4, 8, 0), (8, 8, 4, 1), (4, 4, 8, 1), (6, 6, 3, 0)])
def test_fourier_cn_equals_dense_real_space_cn(oracle_mod, H, W, N, conv):
    """One Crank-Nicolson integration of eq. (4.1) assembled densely in real
    space (no Fourier transform anywhere) equals FFT -> per-frequency CN ->
    iFFT (Theorem 2 states the decoupling is exact)."""
    beta, T, S = 0.7, 0.9, 5
    psi0 = synth.random_real_volume(N, H, W, 3)
    Op = oracle_mod.dense_operator(H, W, N, beta, conv)
    ref = _cn_dense(Op, psi0.ravel(), T, S).reshape(N, H, W)
    got = oracle_mod.inverse(oracle_mod.diffuse(oracle_mod.forward(psi0), beta, T, S, conv))
    np.testing.assert_allclose(got.real, ref, atol=1e-12)
    assert np.abs(got.imag).max() < 1e-12


def test_dense_operator_is_symmetric_generator(oracle_mod):
    """The real-space operator is symmetric (D_x is antisymmetric, L is
    symmetric) and has a zero row sum on constants (mass conservation)."""
    Op = oracle_mod.dense_operator(4, 6, 4, 0.3, 0)
    np.testing.assert_allclose(Op, Op.T, atol=1e-14)
    np.testing.assert_allclose(Op @ np.ones(Op.shape[0]), 0.0, atol=1e-13)


def test_cn_is_second_order_towards_matrix_exponential(oracle_mod):
    """CN converges to e^{T A} (eq. (4.3)) as O(dt^2): halving dt divides
    the error by ~4. The exact propagator is taken from an eigendecomposition
    of the dense real-space operator."""
    H, W, N, beta, T = 6, 6, 4, 0.5, 1.0
    psi0 = synth.random_real_volume(N, H, W, 11)
    Op = oracle_mod.dense_operator(H, W, N, beta, 0)
    exact = _expm_sym(Op, psi0.ravel(), T).reshape(N, H, W)
    errs = []
    for S in (8, 16, 32):
        got = oracle_mod.inverse(oracle_mod.diffuse(oracle_mod.forward(psi0), beta, T, S)).real
        errs.append(np.abs(got - exact).max())
    assert 3.6 < errs[0] / errs[1] < 4.4
    assert 3.6 < errs[1] / errs[2] < 4.4


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------

@pytest.mark.parametrize("N", [3, 8, 16, 33])
def test_zero_frequency_closed_form(oracle_mod, N):
    """At omega = 0 the system is dpsi/dt = beta L psi. L is circulant with
    eigenvalues 2 (cos 2 pi j/N - 1) on the Fourier modes in r, so CN scales
    mode j by ((1 + dt lam_j/2) / (1 - dt lam_j/2))^S, lam_j = 2 beta (cos 2 pi j/N - 1)."""
    beta, T, S = 0.8, 2.0, 37
    v = synth.random_volume(N, 4, 6, 5)
    dt = T / S
    lam = 2.0 * beta * (np.cos(2 * np.pi * np.arange(N) / N) - 1.0)
    rho = ((1 + 0.5 * dt * lam) / (1 - 0.5 * dt * lam)) ** S
    expect = np.fft.ifft(np.fft.fft(v[:, 0, 0]) * rho)
    got = oracle_mod.diffuse(v, beta, T, S)[:, 0, 0]
    np.testing.assert_allclose(got, expect, atol=1e-12)


def test_beta_zero_closed_form(oracle_mod):
    """At beta = 0 the angles decouple: each entry is scaled by
    ((1 - dt a^2/2) / (1 + dt a^2/2))^S with a the DFT symbol, here written
    from the central-difference symbol directly."""
    N, H, W, T, S = 6, 6, 10, 1.5, 9
    v = synth.random_volume(N, H, W, 9)
    dt = T / S
    th = np.pi * np.arange(N) / N
    k = np.arange(H)[None, :, None]
    l = np.arange(W)[None, None, :]
    a = np.cos(th)[:, None, None] * np.sin(2 * np.pi * l / W) + np.sin(th)[:, None, None] * np.sin(2 * np.pi * k / H)
    rho = ((1 - 0.5 * dt * a ** 2) / (1 + 0.5 * dt * a ** 2)) ** S
    np.testing.assert_allclose(oracle_mod.diffuse(v, 0.0, T, S), v * rho, atol=1e-12)


def test_mass_preservation(oracle_mod):
    """The generator has zero row sums (the jump process of Section 2 and
    L 1 = 0), so the total mass sum_{r,x,y} psi is invariant."""
    psi0 = synth.random_real_volume(16, 8, 12, 2)
    out = oracle_mod.inverse(oracle_mod.diffuse(oracle_mod.forward(psi0), 0.6, 3.0, 40)).real
    assert abs(out.sum() - psi0.sum()) < 1e-10 * psi0.sum()


@pytest.mark.parametrize("n", [3, 4, 5, 16, 33, 64])
def test_cyclic_solver_matches_dense_solve(oracle_mod, n):
    """Thomas + Sherman-Morrison equals numpy.linalg.solve on random
    diagonally dominant cyclic tridiagonal systems (the structure the paper
    notes after Theorem 2)."""
    rng = np.random.default_rng(n)
    for off in (-0.3, -1.0, -4.7):
        diag = 2 * abs(off) + rng.uniform(0.01, 3.0, n)
        A = np.diag(diag)
        for i in range(n):
            A[i, (i + 1) % n] += off
            A[i, (i - 1) % n] += off
        b = rng.standard_normal(n)
        np.testing.assert_allclose(oracle_mod.cyclic_solve(diag, off, b), np.linalg.solve(A, b), atol=1e-12)


def test_c_core_matches_dense_per_frequency_solve(oracle_mod):
    v = synth.random_volume(8, 6, 4, 0)
    for conv in (0, 1):
        a = oracle_mod.diffuse(v, 0.7, 0.9, 7, conv)
        b = oracle_mod.diffuse_dense(v, 0.7, 0.9, 7, conv)
        np.testing.assert_allclose(a, b, atol=1e-12)


def test_frequency_subset_leaves_others_untouched(oracle_mod):
    v = synth.random_volume(4, 4, 6, 4)
    full = oracle_mod.diffuse(v, 0.5, 1.0, 10)
    sub = oracle_mod.diffuse(v, 0.5, 1.0, 10, freqs=[0, 5, 23])
    flat_full = full.reshape(4, -1)
    flat_sub = sub.reshape(4, -1)
    flat_v = v.reshape(4, -1)
    for f in range(24):
        ref = flat_full[:, f] if f in (0, 5, 23) else flat_v[:, f]
        np.testing.assert_array_equal(flat_sub[:, f], ref)


# --------------------------------------------------------------------------
# the paper's units (eq. (4.1), eq. (2.14))
# --------------------------------------------------------------------------

@pytest.mark.parametrize("M,N", [(4, 4), (6, 8)])
def test_paper_units_map_exactly(oracle_mod, M, N):
    """(1/2) D of eq. (4.1) (mesh 1/sqrt(M), beta_N) equals (M/2) times the
    pixel-unit operator with beta = beta_N / M, so e^{t_p (1/2) D} is the
    pixel-unit propagator at T = (M/2) t_p; and alpha = beta_N (2 pi/N)^2."""
    alpha, Tp = 0.33, 0.07
    beta, T = oracle_mod.params_from_paper(alpha, Tp, M, N)
    beta_N = beta * M
    assert abs(alpha - beta_N * (2 * np.pi / N) ** 2) < 1e-14
    Dp = oracle_mod.dense_paper_operator(M, N, beta_N)
    Op = oracle_mod.dense_operator(M, M, N, beta, 0)
    np.testing.assert_allclose(Dp, 0.5 * M * Op, atol=1e-12)
    psi0 = synth.random_real_volume(N, M, M, 8).ravel()
    np.testing.assert_allclose(scipy.linalg.expm(Tp * Dp) @ psi0, _expm_sym(Op, psi0, T), atol=1e-10)


def test_table1_parameters_stay_stable(oracle_mod):
    """Every parameter set of Table 1, mapped to pixel units (N=30 as the
    paper uses, M=256), gives a bounded, mass-preserving CN diffusion of one
    restoration interval on a small random volume."""
    rows = [ln.split() for ln in open(__file__.replace("test_oracle_pins.py", "golden/table1.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 13
    psi0 = synth.random_real_volume(30, 8, 8, 1)
    for name, alpha, Tp, n, eps, w, pct in rows:
        beta, T = oracle_mod.params_from_paper(float(alpha), float(Tp), 256, 30)
        out = oracle_mod.inverse(oracle_mod.diffuse(oracle_mod.forward(psi0), beta, T / int(n), 20)).real
        assert np.isfinite(out).all(), name
        assert np.abs(out).max() <= np.abs(psi0).max() * (1 + 1e-9), name
        assert abs(out.sum() - psi0.sum()) < 1e-9 * psi0.sum(), name


# --------------------------------------------------------------------------
# lift and projection
# --------------------------------------------------------------------------

def test_spectral_gradient_of_a_cosine(oracle_mod):
    """Smoothing and differentiation in the DFT domain: for f = 2 + cos(2 pi m x/W)
    the smoothed x-derivative is -(2 pi m/W) exp(-2 pi^2 sigma^2 (m/W)^2) sin(2 pi m x/W),
    and the y-derivative is 0."""
    H, W, m, sigma = 8, 32, 3, 1.3
    x = np.arange(W)
    f = np.tile(2.0 + np.cos(2 * np.pi * m * x / W), (H, 1))
    o = oracle_mod.orient(f, np.ones((H, W), np.uint8), 8, sigma)
    expect = -(2 * np.pi * m / W) * np.exp(-2 * np.pi ** 2 * sigma ** 2 * (m / W) ** 2) * np.sin(2 * np.pi * m * x / W)
    np.testing.assert_allclose(o["gx"], np.tile(expect, (H, 1)), atol=1e-13)
    np.testing.assert_allclose(o["gy"], 0.0, atol=1e-13)


def test_vertical_edge_lifts_to_vertical_direction(oracle_mod):
    """The lift follows the level lines (tangent = gradient + pi/2): a smooth
    vertical ramp has a horizontal gradient, so its pixels go to the bin of
    the vertical direction, th = pi/2, i.e. r = N/2."""
    H, W, N = 16, 32, 8
    x = np.arange(W)
    f = np.tile(1.5 + np.sin(2 * np.pi * x / W), (H, 1))
    o = oracle_mod.orient(f, np.ones((H, W), np.uint8), N)
    moving = np.abs(o["gx"]) > 1e-3 * np.abs(o["gx"]).max()
    assert (o["bins"][moving] == N // 2).all()


def test_flat_image_lifts_to_every_angle(oracle_mod):
    f = np.full((6, 8), 0.4)
    o = oracle_mod.orient(f, np.ones((6, 8), np.uint8), 8)
    assert (o["bins"] == oracle_mod.BIN_FLAT).all()
    vol = oracle_mod.lift(f, np.ones((6, 8), np.uint8), o["bins"], 8)
    np.testing.assert_array_equal(vol.real, np.full((8, 6, 8), 0.4))


def test_project_of_lift_is_identity(oracle_mod):
    w = synth.workload_small(32, 32)
    p = oracle_mod.Params(N=16, beta=0.5, T=1.0, steps=10)
    vol, bins = oracle_mod.lift_from_image(w.f, w.mask, p)
    np.testing.assert_array_equal(oracle_mod.project(vol, 0), w.f)
    single = bins != oracle_mod.BIN_FLAT
    mean = oracle_mod.project(vol, 1)
    np.testing.assert_allclose(mean[single], w.f[single] / 16, rtol=1e-15)
    # exactly one nonzero angle per non-flat known pixel, none on B
    nnz = (vol.real != 0).sum(axis=0)
    assert (nnz[(w.mask == 0)] == 0).all()
    assert (nnz[single & (w.f > 0)] == 1).all()


def _equivariance_inputs(M=24, seed=5):
    clean = synth.lines_circles_image(M, M, seed)
    mask = synth.bernoulli_mask(M, M, seed + 1, 0.3)
    return clean * mask, mask


def _no_ties(oracle_mod, f, mask, N):
    o = oracle_mod.orient(f, mask, N)
    single = o["bins"] != oracle_mod.BIN_FLAT
    assert o["margin"][single].min() > 1e-9
    assert np.abs(o["rel"] - 1e-4).min() > 1e-9


@pytest.mark.parametrize("N", [8, 12])
def test_rotation_by_90_degrees_shifts_channels(oracle_mod, N):
    """Rotating the image by 90 degrees (an exact pixel permutation on the
    periodic grid) rotates the lifted, diffused and restored volume and
    shifts its channels by N/2 (th_r = pi r/N): the discrete form of the
    rotation theorem of Section 3 and of eq. (B.3)."""
    f, mask = _equivariance_inputs()
    _no_ties(oracle_mod, f, mask, N)
    p = oracle_mod.Params(N=N, beta=0.5, T=1.0, steps=8, rounds=2)
    a = oracle_mod.inpaint(f, mask, p, keep=True)
    b = oracle_mod.inpaint(np.rot90(f), np.rot90(mask), p, keep=True)
    rotated = np.stack([np.rot90(a["vol"][(r + N // 2) % N]) for r in range(N)])
    np.testing.assert_allclose(b["vol"].real, rotated.real, atol=1e-12)
    np.testing.assert_allclose(b["out"], np.rot90(a["out"]), atol=1e-12)


def test_flips_map_channels(oracle_mod):
    """A mirror x -> -x maps direction th to pi - th (r -> -r mod N); the
    transpose (x <-> y) maps th to pi/2 - th (r -> N/2 - r mod N)."""
    N = 8
    f, mask = _equivariance_inputs(seed=9)
    _no_ties(oracle_mod, f, mask, N)
    p = oracle_mod.Params(N=N, beta=0.4, T=1.2, steps=6, rounds=2)
    a = oracle_mod.inpaint(f, mask, p, keep=True)
    b = oracle_mod.inpaint(f[:, ::-1], mask[:, ::-1], p, keep=True)
    c = oracle_mod.inpaint(f.T, mask.T, p, keep=True)
    flipped = np.stack([a["vol"][(-r) % N][:, ::-1] for r in range(N)])
    transposed = np.stack([a["vol"][(N // 2 - r) % N].T for r in range(N)])
    np.testing.assert_allclose(b["vol"].real, flipped.real, atol=1e-12)
    np.testing.assert_allclose(c["vol"].real, transposed.real, atol=1e-12)


def test_shift_identity_of_the_appendix(oracle_mod):
    """eq. (B.3): the system at the frequency rotated by 90 degrees is the
    original one conjugated by the channel shift S^{N/2}; so diffusing
    S^{N/2} v at the rotated frequency gives S^{N/2} of the original result."""
    M, N = 12, 8
    v = np.zeros((N, M, M), complex)
    rng = np.random.default_rng(3)
    k, l = 2, 5
    vec = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    v[:, k, l] = vec
    v[:, (-l) % M, k] = np.roll(vec, N // 2)   # frequency (k,l) rotated by 90 degrees
    out = oracle_mod.diffuse(v, 0.9, 1.7, 13)
    np.testing.assert_allclose(out[:, (-l) % M, k], np.roll(out[:, k, l], N // 2), atol=1e-13)


# --------------------------------------------------------------------------
# static restoration
# --------------------------------------------------------------------------

def _mix_case(oracle_mod, N=8, M=16):
    w = synth.workload_small(M, M, seed=4, mask_seed=6)
    o = oracle_mod.orient(w.f, w.mask, N)
    rng = np.random.default_rng(1)
    vol = rng.uniform(0.1, 1.0, (N, M, M)) + 1j * rng.standard_normal((N, M, M)) * 1e-3
    return w, o["bins"], vol


def test_mix_with_eps_one_restores_known_pixels(oracle_mod):
    """eps = 1 makes sigma = h(0)/h(t): the max over angles of every good
    pixel becomes its original value; bad pixels keep their real part."""
    w, bins, vol = _mix_case(oracle_mod)
    out = oracle_mod.mix(vol, w.f, w.mask, bins, 1.0)
    G = w.mask != 0
    np.testing.assert_allclose(out.real.max(axis=0)[G], w.f[G], rtol=1e-14)
    np.testing.assert_array_equal(out.real[:, ~G], vol.real[:, ~G])
    assert (out.imag == 0).all()


def test_mix_with_eps_zero_is_identity(oracle_mod):
    w, bins, vol = _mix_case(oracle_mod)
    out = oracle_mod.mix(vol, w.f, w.mask, bins, 0.0)
    np.testing.assert_allclose(out.real, vol.real, rtol=1e-15)


def test_mix_scales_good_pixels_by_sigma(oracle_mod):
    """Direct check of the SR factor at one pixel with hand-picked values."""
    N = 4
    f = np.array([[0.8]])
    mask = np.array([[1]], np.uint8)
    bins = np.array([[2]], np.uint8)
    vol = np.array([0.1, 0.4, 0.2, -0.3]).reshape(N, 1, 1).astype(complex)
    out = oracle_mod.mix(vol, f, mask, bins, 0.25)
    sigma = (0.25 * 0.8 + 0.75 * 0.4) / 0.4
    np.testing.assert_allclose(out.real.ravel(), sigma * vol.real.ravel(), rtol=1e-15)


def test_mix_relative_guard_blends_linearly(oracle_mod):
    """h(t) = 0.04 <= 0.1 h(0) = 0.08: the division would amplify by ~10,
    so the pixel is blended with its lift instead."""
    N = 4
    f = np.array([[0.8]])
    mask = np.array([[1]], np.uint8)
    bins = np.array([[3]], np.uint8)
    vol = np.array([0.01, 0.04, 0.02, 0.03]).reshape(N, 1, 1).astype(complex)
    out = oracle_mod.mix(vol, f, mask, bins, 0.5, guard=0.1)
    lift = np.array([0.0, 0.0, 0.0, 0.8])
    np.testing.assert_allclose(out.real.ravel(), 0.5 * lift + 0.5 * vol.real.ravel(), rtol=1e-15)
    # just above the threshold the sigma rescaling applies
    vol2 = vol * 2.5   # h(t) = 0.1 > 0.08
    out2 = oracle_mod.mix(vol2, f, mask, bins, 0.5, guard=0.1)
    sigma = (0.5 * 0.8 + 0.5 * 0.1) / 0.1
    np.testing.assert_allclose(out2.real.ravel(), sigma * vol2.real.ravel(), rtol=1e-14)


def test_mix_guard_blends_linearly(oracle_mod):
    N = 4
    f = np.array([[0.8]])
    mask = np.array([[1]], np.uint8)
    bins = np.array([[1]], np.uint8)
    vol = np.array([-0.1, -0.4, -0.2, -0.3]).reshape(N, 1, 1).astype(complex)
    out = oracle_mod.mix(vol, f, mask, bins, 0.5)
    lift = np.array([0.0, 0.8, 0.0, 0.0])
    np.testing.assert_allclose(out.real.ravel(), 0.5 * lift + 0.5 * vol.real.ravel(), rtol=1e-15)


# --------------------------------------------------------------------------
# the whole method
# --------------------------------------------------------------------------

def test_single_round_inpaint_is_lift_diffuse_project(oracle_mod):
    w = synth.workload_small(32, 32)
    p = oracle_mod.Params(N=8, beta=0.5, T=1.0, steps=10, rounds=1)
    res = oracle_mod.inpaint(w.f, w.mask, p)
    vol, bins = oracle_mod.lift_from_image(w.f, w.mask, p)
    manual = oracle_mod.project(oracle_mod.inverse(oracle_mod.diffuse(oracle_mod.forward(vol), 0.5, 1.0, 10)))
    np.testing.assert_array_equal(res["out"], manual)


def test_reinject_keeps_known_pixels_and_fills_the_rest(oracle_mod):
    """The inpainted image (reinject): f itself on every known pixel, and
    on the corrupted ones exactly the plain projection."""
    w = synth.workload_small(32, 32)
    p = oracle_mod.Params(N=8, beta=0.5, T=1.0, steps=10, rounds=2)
    plain = oracle_mod.inpaint(w.f, w.mask, p)["out"]
    p.reinject = 1
    out = oracle_mod.inpaint(w.f, w.mask, p)["out"]
    k = w.mask != 0
    np.testing.assert_array_equal(out[k], w.f[k])
    np.testing.assert_array_equal(out[~k], plain[~k])
    assert np.abs(plain[k] - w.f[k]).max() > 1e-3  # the plain result does move the known pixels


def test_restoration_improves_on_zero_fill_and_beats_downstairs(oracle_mod):
    """Sanity, not parity: on bar-corrupted synthetic data, static
    restoration on the lifted volume brings the corrupted pixels closer to
    the clean image than the zero-filled input, and does clearly better than
    restoring the known pixels on the projected image, the variant the paper
    reports as not working (Section 5, "downstairs or upstairs")."""
    M = 64
    clean = synth.curves_noise_image(M, M, 21, n_curves=10)
    mask = synth.bar_mask(M, M, 3, 12)
    f = clean * mask
    p = oracle_mod.Params(N=16, beta=0.25, T=24.0, steps=20, rounds=6)
    out = oracle_mod.inpaint(f, mask, p)["out"]
    down = oracle_mod.downstairs_restore(f, mask, p)
    B = mask == 0
    err_zero = np.sqrt(np.mean((f[B] - clean[B]) ** 2))
    err_sr = np.sqrt(np.mean((out[B] - clean[B]) ** 2))
    err_down = np.sqrt(np.mean((down[B] - clean[B]) ** 2))
    assert err_sr < 0.75 * err_zero
    assert err_sr < 0.8 * err_down
