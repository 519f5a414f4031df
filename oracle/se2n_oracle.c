/*
 * FP64 CPU oracle for the Mathieu-type diffusion of the SE(2,N) inpainting
 * method. TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU
 * baseline of the benchmark call it; the CUDA library never does.
 *
 * What it computes (Section 4 of the paper, Theorem 2 and eq. (4.2)):
 * after the 2-D DFT of every angle plane, each frequency (k,l) carries an
 * independent N-vector psi that obeys dpsi/dt = A psi with
 *
 *     A = -diag_r(a_r^2) + beta * L,      a_r = wx cos(theta_r) + wy sin(theta_r),
 *     wx = sin(2 pi l / W),  wy = sin(2 pi k / H),
 *
 * L the N x N cyclic second difference (diagonal -2, off-diagonals and the two
 * corners +1). This is eq. (4.2) in pixel units: the exact rescaling of the
 * paper's time and beta_N is done by the Python side (params_from_paper).
 *
 * It is integrated by the Crank-Nicolson scheme the paper recommends
 * (Section 4, remark after Theorem 2, item 2): with dt = T / steps,
 *
 *     (I - dt/2 A) psi_new = (I + dt/2 A) psi_old.
 *
 * The left matrix is tridiagonal plus the two corner entries (the paper
 * notes this structure and points to a dedicated solver); here it is solved
 * the textbook way: Thomas elimination of the tridiagonal part after a
 * Sherman-Morrison split of the corner coupling.
 *
 * Nothing here is blocked, fused or reordered: one frequency at a time, the
 * right-hand side formed explicitly, then the cyclic solve. OpenMP spreads
 * frequencies over host threads (frequencies never interact).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846

/* Solve the tridiagonal system  sub[i] x[i-1] + diag[i] x[i] + sup[i] x[i+1] = rhs[i]
 * (sub[0] and sup[n-1] unused) by Thomas elimination. work has n entries. */
static void thomas(int n, const double *sub, const double *diag, const double *sup,
                   const double *rhs, double *x, double *work) {
    double piv = diag[0];
    x[0] = rhs[0] / piv;
    for (int i = 1; i < n; ++i) {
        work[i] = sup[i - 1] / piv;
        piv = diag[i] - sub[i] * work[i];
        x[i] = (rhs[i] - sub[i] * x[i - 1]) / piv;
    }
    for (int i = n - 2; i >= 0; --i) x[i] -= work[i + 1] * x[i + 1];
}

/* Solve the cyclic tridiagonal system with corner entries
 *   A[0][n-1] = top_corner, A[n-1][0] = bottom_corner
 * by Sherman-Morrison: A = T' + u v^T with u = (g, 0..0, bottom_corner),
 * v = (1, 0..0, top_corner / g), g = -diag[0], T' = A without corners and
 * with diag[0] -> diag[0] - g, diag[n-1] -> diag[n-1] - bottom*top/g.
 * z = T'^{-1} u is passed in precomputed (it depends on the matrix only). */
static void cyclic_solve(int n, const double *sub, const double *diag_mod, const double *sup,
                         double top_corner, double g, const double *z,
                         const double *rhs, double *x, double *work) {
    thomas(n, sub, diag_mod, sup, rhs, x, work);
    const double vx = x[0] + top_corner * x[n - 1] / g;
    const double vz = z[0] + top_corner * z[n - 1] / g;
    const double fact = vx / (1.0 + vz);
    for (int i = 0; i < n; ++i) x[i] -= fact * z[i];
}

/*
 * Integrate `steps` Crank-Nicolson steps of size T/steps for the listed
 * frequencies of the volume vol[N][H][W] (complex128, interleaved re/im),
 * in place. freqs == NULL means every frequency k*W + l. angle_conv 0 puts
 * theta_r = pi r / N (directions), 1 puts theta_r = 2 pi r / N.
 * Returns 0 on success, -1 on bad arguments, -2 on allocation failure.
 */
int se2n_oracle_diffuse(double *vol, int N, int H, int W, double beta, double T, int steps,
                        int angle_conv, const int64_t *freqs, int64_t nfreq, int nthreads) {
    if (!vol || N < 3 || H < 1 || W < 1 || steps < 1 || !(T >= 0.0) || !(beta >= 0.0)) return -1;
    const int64_t HW = (int64_t)H * W;
    const int64_t count = freqs ? nfreq : HW;
    const double dt = T / steps;
    const double step_angle = (angle_conv ? 2.0 : 1.0) * ORACLE_PI / N;
    int failed = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif

#pragma omp parallel
    {
        double *buf = (double *)malloc(sizeof(double) * (size_t)N * 12);
        if (!buf) {
#pragma omp atomic write
            failed = 1;
        }
        double *a2 = buf, *sub = buf + N, *sup = buf + 2 * N, *diag_mod = buf + 3 * N;
        double *z = buf + 4 * N, *u = buf + 5 * N, *work = buf + 6 * N;
        double *re = buf + 7 * N, *im = buf + 8 * N, *rhs = buf + 9 * N, *xs = buf + 10 * N;
#pragma omp for schedule(dynamic, 64)
        for (int64_t t = 0; t < count; ++t) {
            if (!buf) continue;
            const int64_t f = freqs ? freqs[t] : t;
            if (f < 0 || f >= HW) continue;
            const int64_t k = f / W, l = f % W;
            const double wx = sin(2.0 * ORACLE_PI * (double)l / W);
            const double wy = sin(2.0 * ORACLE_PI * (double)k / H);
            for (int r = 0; r < N; ++r) {
                const double a = wx * cos(step_angle * r) + wy * sin(step_angle * r);
                a2[r] = a * a;
            }
            /* Left matrix I - dt/2 A: diagonal 1 + dt/2 (a_r^2 + 2 beta),
             * off-diagonals and corners -dt/2 beta. */
            const double off = -0.5 * dt * beta;
            for (int r = 0; r < N; ++r) {
                sub[r] = off;
                sup[r] = off;
                diag_mod[r] = 1.0 + 0.5 * dt * (a2[r] + 2.0 * beta);
            }
            const double g = -diag_mod[0];
            const double top = off, bottom = off;
            diag_mod[N - 1] -= bottom * top / g;
            diag_mod[0] -= g;
            for (int r = 0; r < N; ++r) u[r] = 0.0;
            u[0] = g;
            u[N - 1] = bottom;
            thomas(N, sub, diag_mod, sup, u, z, work);

            for (int r = 0; r < N; ++r) {
                re[r] = vol[2 * ((int64_t)r * HW + f)];
                im[r] = vol[2 * ((int64_t)r * HW + f) + 1];
            }
            for (int s = 0; s < steps; ++s) {
                double *comp[2] = {re, im};
                for (int c = 0; c < 2; ++c) {
                    double *p = comp[c];
                    /* right-hand side (I + dt/2 A) psi */
                    for (int r = 0; r < N; ++r) {
                        const double left = p[(r + N - 1) % N], right = p[(r + 1) % N];
                        rhs[r] = p[r] + 0.5 * dt * (-a2[r] * p[r] + beta * (left - 2.0 * p[r] + right));
                    }
                    cyclic_solve(N, sub, diag_mod, sup, top, g, z, rhs, xs, work);
                    memcpy(p, xs, sizeof(double) * N);
                }
            }
            for (int r = 0; r < N; ++r) {
                vol[2 * ((int64_t)r * HW + f)] = re[r];
                vol[2 * ((int64_t)r * HW + f) + 1] = im[r];
            }
        }
        free(buf);
    }
    return failed ? -2 : 0;
}

/* Stand-alone cyclic tridiagonal solve (constant off-diagonal `off` on both
 * sides and in both corners, diagonal `diag`), exposed so the tests can pin
 * the solver against a dense solve. Returns 0, or -1 on bad arguments. */
int se2n_oracle_cyclic_solve(int n, const double *diag, double off, const double *rhs, double *x) {
    if (n < 3 || !diag || !rhs || !x) return -1;
    double *buf = (double *)malloc(sizeof(double) * (size_t)n * 6);
    if (!buf) return -2;
    double *sub = buf, *sup = buf + n, *dm = buf + 2 * n, *z = buf + 3 * n, *u = buf + 4 * n, *work = buf + 5 * n;
    for (int i = 0; i < n; ++i) {
        sub[i] = off;
        sup[i] = off;
        dm[i] = diag[i];
        u[i] = 0.0;
    }
    const double g = -diag[0];
    dm[n - 1] -= off * off / g;
    dm[0] -= g;
    u[0] = g;
    u[n - 1] = off;
    thomas(n, sub, dm, sup, u, z, work);
    cyclic_solve(n, sub, dm, sup, off, g, z, rhs, x, work);
    free(buf);
    return 0;
}
