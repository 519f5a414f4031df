"""Plant plausible mistakes in the oracle (on the CPU, by monkeypatching the
oracle module) and check that the pins of test_oracle_pins.py catch each one.

A pin that no mistake can fail pins nothing; this file shows each pinned
stage has teeth.
"""
import numpy as np
import pytest

import oracle
import test_oracle_pins as pins


def _mutant_diffuse(kind):
    """A Crank-Nicolson diffusion in plain numpy with one planted slip."""

    def run(vol_hat, beta, T, steps, angle_conv=0, freqs=None, nthreads=0):
        v = np.array(vol_hat, dtype=np.complex128, copy=True)
        N, H, W = v.shape
        th = (2.0 if (angle_conv or kind == "angle_2pi") else 1.0) * np.pi * np.arange(N) / N
        wx = np.sin(2 * np.pi * np.arange(W) / W)
        wy = np.sin(2 * np.pi * np.arange(H) / H)
        if kind == "swap_axes":
            wx = np.sin(2 * np.pi * np.arange(W) / H) if H != W else np.sin(2 * np.pi * np.arange(W) / W) * 0.9
            wy = np.sin(2 * np.pi * np.arange(H) / W) if H != W else np.sin(2 * np.pi * np.arange(H) / H) * 1.1
        b = beta * (0.5 if kind == "half_beta" else 1.0)
        dt = T / steps * (2.0 if kind == "double_dt" else 1.0)
        L = -2.0 * np.eye(N)
        for r in range(N):
            L[r, (r + 1) % N] += 1.0
            L[r, (r - 1) % N] += 1.0
        if kind == "no_corners":
            L[0, N - 1] -= 1.0
            L[N - 1, 0] -= 1.0
        I = np.eye(N)
        for k in range(H):
            for l in range(W):
                a = wx[l] * np.cos(th) + wy[k] * np.sin(th)
                A = -np.diag(a ** 2) + b * L
                if kind == "euler":
                    step = I + dt * A
                else:
                    step = np.linalg.solve(I - 0.5 * dt * A, I + 0.5 * dt * A)
                for _ in range(steps):
                    v[:, k, l] = step @ v[:, k, l]
        return v

    return run


def _caught(fn, *args):
    try:
        fn(*args)
    except AssertionError:
        return True
    return False


def _diffusion_pins_catch(monkeypatch, kind):
    monkeypatch.setattr(oracle, "diffuse", _mutant_diffuse(kind))
    checks = [
        lambda: pins.test_fourier_cn_equals_dense_real_space_cn(oracle, 4, 6, 4, 0),
        lambda: pins.test_fourier_cn_equals_dense_real_space_cn(oracle, 6, 6, 3, 0),
        lambda: pins.test_cn_is_second_order_towards_matrix_exponential(oracle),
        lambda: pins.test_zero_frequency_closed_form(oracle, 8),
        lambda: pins.test_mass_preservation(oracle),
        lambda: pins.test_shift_identity_of_the_appendix(oracle),
    ]
    return [_caught(c) for c in checks]


def test_unmutated_python_cn_passes_every_diffusion_pin(monkeypatch):
    assert not any(_diffusion_pins_catch(monkeypatch, "none"))


@pytest.mark.parametrize("kind", ["swap_axes", "half_beta", "double_dt", "no_corners", "euler", "angle_2pi"])
def test_planted_diffusion_mistake_is_caught(monkeypatch, kind):
    assert any(_diffusion_pins_catch(monkeypatch, kind)), kind


def test_swapped_symbol_axes_are_caught(monkeypatch):
    real = oracle.omegas
    monkeypatch.setattr(oracle, "omegas", lambda H, W: real(W, H)[::-1] if H == W else
                        (np.sin(2 * np.pi * np.arange(W) / H), np.sin(2 * np.pi * np.arange(H) / W)))
    assert _caught(pins.test_central_difference_symbol, oracle, 6, 10)


def test_wrong_angle_grid_breaks_rotation_equivariance(monkeypatch):
    """Lift bins taken on a 2 pi/N grid while the operator uses pi/N."""
    real_orient = oracle.orient

    def orient_2pi(f, mask, N, sigma=1.0, angle_conv=0, flat_tol=1e-4):
        return real_orient(f, mask, N, sigma, 1, flat_tol)

    monkeypatch.setattr(oracle, "orient", orient_2pi)
    assert _caught(pins.test_rotation_by_90_degrees_shifts_channels, oracle, 8)


def test_gradient_instead_of_tangent_is_caught(monkeypatch):
    real_orient = oracle.orient

    def orient_grad(f, mask, N, sigma=1.0, angle_conv=0, flat_tol=1e-4):
        o = real_orient(f, mask, N, sigma, angle_conv, flat_tol)
        flat = o["bins"] == oracle.BIN_FLAT
        b = (o["bins"].astype(int) + N // 2) % N
        o["bins"] = np.where(flat, oracle.BIN_FLAT, b).astype(np.uint8)
        return o

    monkeypatch.setattr(oracle, "orient", orient_grad)
    assert _caught(pins.test_vertical_edge_lifts_to_vertical_direction, oracle)


def test_dropped_gaussian_is_caught(monkeypatch):
    real_orient = oracle.orient

    def orient_sharp(f, mask, N, sigma=1.0, angle_conv=0, flat_tol=1e-4):
        return real_orient(f, mask, N, 0.0, angle_conv, flat_tol)

    monkeypatch.setattr(oracle, "orient", orient_sharp)
    assert _caught(pins.test_spectral_gradient_of_a_cosine, oracle)


def test_swapped_restoration_factor_is_caught(monkeypatch):
    real_mix = oracle.mix

    def mix_swapped(vol, f, mask, bins, eps, guard=1e-12):
        # sigma = (eps h(t) + (1-eps) h(0)) / h(t): eps applied to the wrong term
        return real_mix(vol, f, mask, bins, 1.0 - eps, guard)

    monkeypatch.setattr(oracle, "mix", mix_swapped)
    assert _caught(pins.test_mix_scales_good_pixels_by_sigma, oracle)
    assert _caught(pins.test_mix_with_eps_one_restores_known_pixels, oracle)


def test_wrong_paper_time_scale_is_caught(monkeypatch):
    real = oracle.params_from_paper
    monkeypatch.setattr(oracle, "params_from_paper",
                        lambda a, T, M, N: (real(a, T, M, N)[0], real(a, T, M, N)[1] * 2))
    assert _caught(pins.test_paper_units_map_exactly, oracle, 4, 4)
