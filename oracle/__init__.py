"""FP64 CPU oracle for the SE(2,N) hypoelliptic-diffusion inpainting path.

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. It shares no code
with the CUDA library and never touches a GPU.

It restates, step by step and in float64 / complex128, what the paper's
method computes (Boscain, Chertovskih, Gauthier, Remizov, "Hypoelliptic
diffusion and human vision: a semi-discrete new twist"):

* lift            -- Section 1.2.4 (first item): Gaussian smoothing and the
                     gradient both taken in the FFT domain, each pixel lifted
                     to the closest discrete direction;
* forward/inverse -- Theorem 2: 2-D DFT of every angle plane;
* diffuse         -- eq. (4.2) integrated by Crank-Nicolson (Section 4,
                     remark after Theorem 2), see se2n_oracle.c;
* mix             -- static restoration (Section 5, "Static restoration"):
                     sigma = (eps h(0) + (1-eps) h(t_i)) / h(t_i) on the good set;
* dr_grow         -- dynamic restoration (Section 5.3): the good set grows
                     into the corrupted one from its boundary;
* project         -- Section 1.2.4 (second item): maximum (default) or mean
                     over the angles;
* inpaint         -- the whole method: lift, then n restoration intervals.

Canonical units. The operator is written in pixel units,
    dpsi_r/dt = (cos th_r Dx + sin th_r Dy)^2 psi_r + beta (psi_{r-1} - 2 psi_r + psi_{r+1}),
with Dx, Dy the periodic central differences (psi[x+1]-psi[x-1])/2, so the
DFT symbol of the first term is -a_r^2 with a_r = wx cos th_r + wy sin th_r,
wx = sin(2 pi l/W), wy = sin(2 pi k/H). The paper's eq. (4.1) uses the mesh
step 1/sqrt(M) and a factor 1/2; params_from_paper maps its (alpha, T) onto
this form exactly.

Readings taken where the paper is silent:
  * th_r = pi r / N (directions, the projectivised picture) by default,
    2 pi r / N on request (angle_conv=1);
  * the lift goes to the level-line tangent (gradient angle + pi/2), the
    lifted value is the unsmoothed f, the Gaussian has sigma = 1 px;
  * a pixel whose smoothed gradient is below flat_tol * max|grad| is "flat"
    and is lifted to every angle;
  * the image is zero on the corrupted set B (f = f * mask);
  * restoration divides by h(t_i) only where h(t_i) > guard * h(0) (guard =
    0.1, so sigma <= 5.5 for eps = 0.5); elsewhere the good pixel is mixed
    linearly with its lift;
  * dynamic restoration tests the current image h(t_i) = max over angles
    before the restoration at t_i; the boundary of B is the set of bad pixels
    with a good 8-neighbour; the mean runs over the bad pixels of the 3x3
    block inside the image (the pixel included); the comparison is strict;
    every pixel decides on the sets before the step; a pixel that joins is
    restored from then on like a known pixel of value h(t_i) lifted to the
    angle of its largest value (the first one on ties).

Every function here is pinned by a test under tests/ against a closed form,
a dense brute-force computation, an invariant or a textbook routine.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import numpy as np

from . import build as _build

BIN_FLAT = 255

__all__ = [
    "BIN_FLAT", "Params", "angles", "omegas", "symbol", "params_from_paper",
    "orient", "lift", "lift_from_image", "forward", "inverse", "diffuse",
    "diffuse_dense", "cyclic_solve", "mix", "dr_grow", "project", "inpaint",
    "downstairs_restore", "dense_operator", "dense_paper_operator", "rel_l2",
]


@dataclasses.dataclass
class Params:
    """Method parameters (pixel units). T is the total time over all rounds;
    each of the `rounds` restoration intervals integrates T/rounds in
    `steps` Crank-Nicolson steps."""

    N: int
    beta: float
    T: float
    steps: int
    rounds: int = 1
    eps: float = 0.5
    sigma: float = 1.0
    proj: int = 0            # 0 = max over angles, 1 = mean
    angle_conv: int = 0      # 0: th_r = pi r/N, 1: th_r = 2 pi r/N
    flat_tol: float = 1e-4
    final_mix: int = 0       # 1: restore once more after the last interval
    guard: float = 0.1       # relative: sigma only where h(t) > guard * h(0)
    reinject: int = 0        # 1: the result keeps f on the known pixels (the inpainted image)
    dynamic: int = 0         # 1: dynamic restoration (Section 5.3): the good set grows each round


# ----------------------------------------------------------------------------
# the C core
# ----------------------------------------------------------------------------

_lib = None


def _clib():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        lib.se2n_oracle_diffuse.restype = ctypes.c_int
        lib.se2n_oracle_diffuse.argtypes = [
            ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
            ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64,
            ctypes.c_int]
        lib.se2n_oracle_cyclic_solve.restype = ctypes.c_int
        lib.se2n_oracle_cyclic_solve.argtypes = [
            ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
        _lib = lib
    return _lib


# ----------------------------------------------------------------------------
# grids and symbols
# ----------------------------------------------------------------------------

def angles(N: int, angle_conv: int = 0) -> np.ndarray:
    """Discrete angles th_r, r = 0..N-1 (pi r/N, or 2 pi r/N)."""
    return (2.0 if angle_conv else 1.0) * np.pi * np.arange(N) / N


def omegas(H: int, W: int):
    """Central-difference symbols: wx[l] = sin(2 pi l/W), wy[k] = sin(2 pi k/H)
    (Theorem 2: the DFT maps D_x to multiplication by i sin(2 pi (k-1)/M),
    written here with zero-based indices and unit mesh step)."""
    return np.sin(2.0 * np.pi * np.arange(W) / W), np.sin(2.0 * np.pi * np.arange(H) / H)


def symbol(H: int, W: int, N: int, angle_conv: int = 0) -> np.ndarray:
    """a[r][k][l] = wx[l] cos th_r + wy[k] sin th_r (Theorem 2, a^r_{k,l})."""
    wx, wy = omegas(H, W)
    th = angles(N, angle_conv)
    return (np.cos(th)[:, None, None] * wx[None, None, :]
            + np.sin(th)[:, None, None] * wy[None, :, None])


def params_from_paper(alpha: float, T_paper: float, M: int, N: int):
    """Map the paper's (alpha, T) on an M x M image to pixel units.

    eq. (2.14): alpha = beta_N (2 pi / N)^2. eq. (4.1) has mesh step
    1/sqrt(M) and the factor 1/2, so in the paper's time t_p the system reads
    dpsi/dt_p = (M/2) [ -a^2 psi + (beta_N/M) L psi ]; with t = (M/2) t_p it is
    the pixel-unit form with beta = beta_N / M.
    Returns (beta, T)."""
    beta_N = alpha * (N / (2.0 * np.pi)) ** 2
    return beta_N / M, 0.5 * M * T_paper


# ----------------------------------------------------------------------------
# lift and projection
# ----------------------------------------------------------------------------

def _signed(n: int) -> np.ndarray:
    """Signed DFT frequencies 0, 1, ..., n/2-1, -n/2, ..., -1."""
    return np.fft.fftfreq(n) * n


def orient(f, mask, N, sigma=1.0, angle_conv=0, flat_tol=1e-4):
    """Direction bin of every pixel (Section 1.2.4, first item).

    The image (zero on B) is smoothed by a Gaussian of sigma px and
    differentiated, both in the DFT domain; the tangent direction
    phi = atan2(gy, gx) + pi/2 (mod pi) goes to the closest discrete angle
    bin = floor(phi / dth + 1/2) mod N. Flat pixels get BIN_FLAT.

    Returns a dict with bins (uint8), gx, gy, phi, margin (distance of
    phi/dth + 1/2 to the nearest integer, in bins) and rel (|grad| / max|grad|)."""
    f = np.asarray(f, dtype=np.float64)
    H, W = f.shape
    f0 = f * (np.asarray(mask) != 0)
    F = np.fft.fft2(f0)
    kt = _signed(H)[:, None]
    lt = _signed(W)[None, :]
    G = np.exp(-2.0 * np.pi ** 2 * sigma ** 2 * ((kt / H) ** 2 + (lt / W) ** 2))
    ddx = 2j * np.pi * lt / W
    ddy = 2j * np.pi * kt / H
    ddx = np.where(lt == -W / 2, 0.0, ddx)   # the Nyquist column has no sign: no derivative
    ddy = np.where(kt == -H / 2, 0.0, ddy)
    gx = np.fft.ifft2(F * G * ddx).real
    gy = np.fft.ifft2(F * G * ddy).real
    mag = np.hypot(gx, gy)
    gmax = mag.max()
    rel = mag / gmax if gmax > 0 else np.zeros_like(mag)
    flat = rel <= flat_tol
    phi = np.mod(np.arctan2(gy, gx) + 0.5 * np.pi, np.pi)
    dth = (2.0 if angle_conv else 1.0) * np.pi / N
    u = phi / dth + 0.5
    bins = np.mod(np.floor(u), N).astype(np.int64)
    frac = u - np.floor(u)
    margin = np.minimum(frac, 1.0 - frac)
    bins = np.where(flat, BIN_FLAT, bins).astype(np.uint8)
    return dict(bins=bins, gx=gx, gy=gy, phi=phi, margin=margin, rel=rel)


def lift(f, mask, bins, N):
    """Lifted volume psi[r][y][x] = f(x,y) if r is the pixel's bin (every r
    for a flat pixel), else 0; f is zero on B. complex128 [N][H][W]."""
    f0 = np.asarray(f, dtype=np.float64) * (np.asarray(mask) != 0)
    bins = np.asarray(bins)
    r = np.arange(N)[:, None, None]
    on = (bins[None] == r) | (bins[None] == BIN_FLAT)
    return np.where(on, f0[None], 0.0).astype(np.complex128)


def lift_from_image(f, mask, p: Params):
    o = orient(f, mask, p.N, p.sigma, p.angle_conv, p.flat_tol)
    return lift(f, mask, o["bins"], p.N), o["bins"]


def project(vol, proj=0):
    """Back to the image (Section 1.2.4, second item): max over angles of the
    real part (proj=0), or the mean (proj=1)."""
    re = np.asarray(vol).real
    return re.max(axis=0) if proj == 0 else re.mean(axis=0)


# ----------------------------------------------------------------------------
# transforms and diffusion
# ----------------------------------------------------------------------------

def forward(vol):
    """Unnormalised 2-D DFT of every angle plane (Theorem 2)."""
    return np.fft.fft2(np.asarray(vol, dtype=np.complex128), axes=(1, 2))


def inverse(vol_hat):
    """Inverse 2-D DFT of every angle plane, including 1/(H W)."""
    return np.fft.ifft2(np.asarray(vol_hat, dtype=np.complex128), axes=(1, 2))


def diffuse(vol_hat, beta, T, steps, angle_conv=0, freqs=None, nthreads=0):
    """Crank-Nicolson integration of eq. (4.2) over time T in `steps`
    steps, for every frequency (or only the flat indices k*W+l in freqs;
    other frequencies are returned unchanged). Returns a new array."""
    v = np.array(vol_hat, dtype=np.complex128, order="C", copy=True)
    N, H, W = v.shape
    if freqs is not None:
        fr = np.ascontiguousarray(np.asarray(freqs, dtype=np.int64))
        ptr, n = fr.ctypes.data, fr.size
    else:
        fr, ptr, n = None, None, 0
    rc = _clib().se2n_oracle_diffuse(v.ctypes.data, N, H, W, float(beta), float(T), int(steps),
                                     int(angle_conv), ptr, n, int(nthreads))
    if rc != 0:
        raise ValueError(f"oracle diffuse failed with code {rc}")
    return v


def cyclic_solve(diag, off, rhs):
    """Cyclic tridiagonal solve (diagonal `diag`, off-diagonals and corners
    `off`) by the C core's Thomas + Sherman-Morrison routine."""
    d = np.ascontiguousarray(np.asarray(diag, dtype=np.float64))
    b = np.ascontiguousarray(np.asarray(rhs, dtype=np.float64))
    x = np.empty_like(b)
    rc = _clib().se2n_oracle_cyclic_solve(d.size, d.ctypes.data, float(off), b.ctypes.data, x.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle cyclic solve failed with code {rc}")
    return x


def _cyclic_laplacian(N):
    L = -2.0 * np.eye(N)
    for r in range(N):
        L[r, (r - 1) % N] += 1.0
        L[r, (r + 1) % N] += 1.0
    return L


def diffuse_dense(vol_hat, beta, T, steps, angle_conv=0):
    """The same Crank-Nicolson integration with a dense N x N solve per
    frequency (numpy.linalg.solve). Small sizes only; used to pin the C core."""
    v = np.array(vol_hat, dtype=np.complex128, copy=True)
    N, H, W = v.shape
    a = symbol(H, W, N, angle_conv)
    L = _cyclic_laplacian(N)
    dt = T / steps
    I = np.eye(N)
    for k in range(H):
        for l in range(W):
            A = -np.diag(a[:, k, l] ** 2) + beta * L
            step = np.linalg.solve(I - 0.5 * dt * A, I + 0.5 * dt * A)
            psi = v[:, k, l]
            for _ in range(steps):
                psi = step @ psi
            v[:, k, l] = psi
    return v


# ----------------------------------------------------------------------------
# static restoration
# ----------------------------------------------------------------------------

def mix(vol, f, mask, bins, eps, guard=0.1, ht=None, h0=None):
    """Static restoration at the good pixels (Section 5, SR).

    h(t) = max over angles of the current volume, h(0) = max over angles of
    the lift; on G every angle is scaled by
    sigma = (eps h(0) + (1-eps) h(t)) / h(t). Where h(t) <= guard * h(0) (or
    h(t) <= 0) the division would amplify the small residual by more than
    eps/guard, and the good pixel is instead set to eps * lift + (1-eps) * psi,
    which moves its maximum to about the same eps h(0) + (1-eps) h(t). The
    volume is real (the imaginary part is dropped everywhere); B pixels are
    otherwise unchanged.

    ht, h0 (optional): h(t) and h(0) given instead of taken over the planes
    of vol, for a volume that holds only some of the angles (bins then
    number the planes of vol; a pixel lifted elsewhere names none of them)."""
    re = np.asarray(vol).real.copy()
    N = re.shape[0]
    psi0 = lift(f, mask, bins, N).real
    h0 = psi0.max(axis=0) if h0 is None else np.asarray(h0, dtype=np.float64)
    ht = re.max(axis=0) if ht is None else np.asarray(ht, dtype=np.float64)
    good = np.asarray(mask) != 0
    scaled = good & (ht > guard * h0) & (ht > 0.0)
    lin = good & ~scaled
    sig = np.ones_like(ht)
    sig[scaled] = (eps * h0[scaled] + (1.0 - eps) * ht[scaled]) / ht[scaled]
    out = re * sig[None]
    out[:, lin] = eps * psi0[:, lin] + (1.0 - eps) * re[:, lin]
    return out.astype(np.complex128)


def dr_grow(vol, mask, fref, bins, dtype=np.float64, return_margin=False):
    """One step of dynamic restoration (Section 5.3): the good set G_i is
    G_{i-1} plus every pixel of the boundary of B_{i-1} whose image value
    exceeds the mean of the image over the pixels of B_{i-1} in its 3x3
    neighbourhood.

    vol: the volume at the restoration time (its real part is used); mask,
    fref, bins: the good set (nonzero = good) and, for its pixels, the
    reference value and orientation bin that the restoration pulls them to.
    The image is h = max over angles. A bad pixel is on the boundary when one
    of its 8 neighbours is good; its mean runs over the bad pixels of its 3x3
    block (itself included) that lie inside the image, summed row by row,
    top to bottom and left to right, and it joins when h > sum / count.
    Decisions use the sets before the step. A joining pixel gets fref = h and
    bins = the angle of its largest value (the first on ties).

    dtype: precision of h, the sums and the comparison; float32 takes the
    decision the way an FP32 kernel summing in the same order does.

    Returns (mask, fref, bins) of G_i as new arrays, and with return_margin
    also the map of |h - mean| over the boundary pixels whose block holds
    another bad pixel (inf elsewhere): how far each decision that rounding
    could change is from a tie. A pixel whose 8 neighbours are all good
    compares h with itself and never joins, in any precision."""
    re = np.asarray(vol).real.astype(dtype)
    h = re.max(axis=0)
    amax = np.argmax(re, axis=0).astype(np.uint8)
    good = np.asarray(mask) != 0
    bad = ~good
    H, W = h.shape
    acc = np.zeros((H, W), dtype=dtype)
    cnt = np.zeros((H, W), dtype=np.int64)
    boundary = np.zeros((H, W), dtype=bool)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            # neighbour (y + dy, x + dx) of every pixel (y, x) that has one
            ys = slice(max(0, -dy), H - max(0, dy))
            xs = slice(max(0, -dx), W - max(0, dx))
            ny = slice(max(0, dy), H + min(0, dy))
            nx = slice(max(0, dx), W + min(0, dx))
            nb_bad = bad[ny, nx]
            acc[ys, xs] = np.where(nb_bad, acc[ys, xs] + h[ny, nx], acc[ys, xs])
            cnt[ys, xs] += nb_bad
            if dy or dx:
                boundary[ys, xs] |= good[ny, nx]
    mean = np.divide(acc, cnt.astype(dtype), out=np.zeros_like(acc), where=cnt > 0)
    join = bad & boundary & (h > mean)
    new_mask = np.where(join, 1, good.astype(np.uint8)).astype(np.uint8)
    new_fref = np.where(join, h.astype(np.float64), np.asarray(fref, dtype=np.float64))
    new_bins = np.where(join, amax, np.asarray(bins)).astype(np.uint8)
    if return_margin:
        cand = bad & boundary & (cnt >= 2)
        margin = np.where(cand, np.abs(h - mean).astype(np.float64), np.inf)
        return new_mask, new_fref, new_bins, margin
    return new_mask, new_fref, new_bins


# ----------------------------------------------------------------------------
# the whole method
# ----------------------------------------------------------------------------

def inpaint(f, mask, p: Params, bins=None, nthreads=0, keep=False, tie_tol=0.0, store=None):
    """Lift, then `rounds` intervals of length T/rounds: the first starts
    from the lift; each later one starts from the statically restored state
    (the mix at t_0 is the identity, sigma = 1). The state at T is inverted
    and projected (mixed once more first if final_mix). With reinject the
    known pixels of the result are f itself: the method only fills the
    corrupted ones.

    With dynamic, every restoration is preceded by one growth step of the
    good set (dr_grow); reinject still keeps only the given known pixels.

    Returns a dict with out (the image), bins, the final good set (mask_final,
    equal to the given one without dynamic), the smallest decision margin of
    the growth steps (dr_margin, inf without dynamic), the pixels whose
    decision came within tie_tol of a tie in some growth step (dr_ties) and,
    if keep, the final volume.

    store: a function applied to the volume at every point where an
    implementation of the method keeps it in memory between two stages
    (after the lift, each transform, each diffusion and each restoration);
    None is the identity. Rounding it to complex64 there measures how far
    FP32 storage alone moves the FP64 result (the sensitivity that bounds
    any FP32 implementation from below); it changes no arithmetic of the
    method."""
    if bins is None:
        bins = orient(f, mask, p.N, p.sigma, p.angle_conv, p.flat_tol)["bins"]
    g_mask = (np.asarray(mask) != 0).astype(np.uint8)
    g_fref = np.asarray(f, dtype=np.float64) * g_mask
    g_bins = np.asarray(bins).astype(np.uint8)
    margin = float("inf")
    ties = np.zeros(g_mask.shape, dtype=bool)

    def restore(v):
        nonlocal g_mask, g_fref, g_bins, margin, ties
        if p.dynamic:
            g_mask, g_fref, g_bins, m = dr_grow(v, g_mask, g_fref, g_bins, return_margin=True)
            margin = min(margin, float(m.min()))
            ties |= m < tie_tol
        return mix(v, g_fref, g_mask, g_bins, p.eps, p.guard)

    st = store if store is not None else (lambda x: x)
    Tr = p.T / p.rounds
    v = st(forward(st(lift(f, mask, bins, p.N))))
    v = st(diffuse(v, p.beta, Tr, p.steps, p.angle_conv, nthreads=nthreads))
    for _ in range(1, p.rounds):
        v = st(restore(st(inverse(v))))
        v = st(diffuse(st(forward(v)), p.beta, Tr, p.steps, p.angle_conv, nthreads=nthreads))
    v = st(inverse(v))
    if p.final_mix:
        v = st(restore(v))
    out = project(v, p.proj)
    if p.reinject:
        out = np.where(np.asarray(mask) != 0, np.asarray(f, dtype=np.float64), out)
    res = dict(out=out, bins=bins, mask_final=g_mask, dr_margin=margin, dr_ties=ties)
    if keep:
        res["vol"] = v
    return res


def downstairs_restore(f, mask, p: Params, nthreads=0):
    """The image-level restoration the paper tries first and rejects
    (Section 5, "Restoration: downstairs or upstairs?"): lift, diffuse over
    T/rounds, project, put the known pixels back, repeat. Negative control."""
    g = np.asarray(f, dtype=np.float64) * (np.asarray(mask) != 0)
    known = np.asarray(mask) != 0
    Tr = p.T / p.rounds
    for _ in range(p.rounds):
        bins = orient(g, np.ones_like(mask), p.N, p.sigma, p.angle_conv, p.flat_tol)["bins"]
        v = diffuse(forward(lift(g, np.ones_like(mask), bins, p.N)), p.beta, Tr, p.steps,
                    p.angle_conv, nthreads=nthreads)
        img = project(inverse(v), p.proj)
        g = np.where(known, f, img)
    return g


# ----------------------------------------------------------------------------
# dense real-space operators (brute force, tiny grids only)
# ----------------------------------------------------------------------------

def _central_diff(n, step=1.0):
    D = np.zeros((n, n))
    for i in range(n):
        D[i, (i + 1) % n] += 0.5 / step
        D[i, (i - 1) % n] -= 0.5 / step
    return D


def dense_operator(H, W, N, beta, angle_conv=0):
    """The fully discrete operator of eq. (4.1) in pixel units, assembled in
    real space without any Fourier transform: block r is
    (cos th_r Dx + sin th_r Dy)^2 with periodic central differences, plus
    beta * (L kron I). Index order r*H*W + y*W + x. Size (N H W)^2."""
    Dx = np.kron(np.eye(H), _central_diff(W))
    Dy = np.kron(_central_diff(H), np.eye(W))
    th = angles(N, angle_conv)
    HW = H * W
    Op = np.zeros((N * HW, N * HW))
    for r in range(N):
        Dr = np.cos(th[r]) * Dx + np.sin(th[r]) * Dy
        Op[r * HW:(r + 1) * HW, r * HW:(r + 1) * HW] = Dr @ Dr
    Op += beta * np.kron(_cyclic_laplacian(N), np.eye(HW))
    return Op


def dense_paper_operator(M, N, beta_N):
    """The right-hand side (1/2) D of eq. (4.1) in the paper's own units on
    an M x M grid: mesh step 1/sqrt(M), differences (sqrt(M)/2)(psi_{k+1} -
    psi_{k-1}), angular term beta_N (psi^{r-1} - 2 psi^r + psi^{r+1}),
    directions e_r = pi r / N."""
    s = 1.0 / np.sqrt(M)
    Dx = np.kron(np.eye(M), _central_diff(M, step=s))
    Dy = np.kron(_central_diff(M, step=s), np.eye(M))
    th = angles(N, 0)
    HW = M * M
    D = np.zeros((N * HW, N * HW))
    for r in range(N):
        Dr = np.cos(th[r]) * Dx + np.sin(th[r]) * Dy
        D[r * HW:(r + 1) * HW, r * HW:(r + 1) * HW] = Dr @ Dr
    D += beta_N * np.kron(_cyclic_laplacian(N), np.eye(HW))
    return 0.5 * D


def rel_l2(x, ref):
    """||x - ref||_2 / ||ref||_2 over all elements."""
    x = np.asarray(x)
    ref = np.asarray(ref)
    den = np.linalg.norm(ref.ravel())
    return float(np.linalg.norm((x - ref).ravel()) / (den if den > 0 else 1.0))
