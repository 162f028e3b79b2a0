/*
 * kde_oracle.c -- plain, slow, FP64 CPU oracle for the KDE-PIC hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * Everything here is the plain definition written out in double precision:
 * dense sums over all (particle, node) and (particle, particle) pairs, no
 * truncation, no sorting, no fixed-point positions (x is a double in [0, L)).
 * Outer loops are split across OpenMP threads; every sum over an inner index
 * runs in index order inside one thread, and per-row results are combined in
 * row order afterwards, so results do not depend on the thread count.
 *
 * Paper: Wu & Qin, "Reducing Noise for PIC Simulations Using Kernel Density
 * Estimation Algorithm" (arXiv 1804.11174).
 *
 * Conventions: theta = 2 pi x / L maps the periodic domain onto the circle.
 * Densities in theta units integrate to 1 over [0, 2pi); a density in x units
 * is (2 pi / L) times the theta-unit density.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_TWO_PI 6.283185307179586476925286766559
#define OR_PI 3.1415926535897932384626433832795

/* ------------------------------------------------------------------------ */
/* Sec. II.A, Eq. (vonMises): normalisation by the modified Bessel function  */
/* I0.  The oracle uses the scaled function I0e(x) = exp(-x) I0(x) so that   */
/* exp(kappa cos t) / I0(kappa) = exp(kappa (cos t - 1)) / I0e(kappa) never  */
/* overflows.  Power series for x < 30, the Hankel asymptotic expansion      */
/* (Abramowitz & Stegun 9.7.1, all terms positive for order 0) above.        */
/* ------------------------------------------------------------------------ */
double or_i0e(double x)
{
    if (x < 0) x = -x;
    if (x < 30.0) {
        /* I0(x) = sum_k ((x/2)^k / k!)^2 */
        double q = 0.25 * x * x, term = 1.0, sum = 1.0;
        for (int k = 1; k < 1000; ++k) {
            term *= q / ((double)k * (double)k);
            sum += term;
            if (term < 1e-18 * sum) break;
        }
        return sum * exp(-x);
    }
    /* I0(x) ~ e^x / sqrt(2 pi x) * sum_k prod_{j<=k} (2j-1)^2 / (8 x j) */
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 400; ++k) {
        double next = term * (2.0 * k - 1.0) * (2.0 * k - 1.0) / (8.0 * x * k);
        if (next >= term) break; /* asymptotic series: stop at the smallest term */
        term = next;
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return sum / sqrt(OR_TWO_PI * x);
}

/* Eq. (vonMises) with mu = 0: K_kappa(t) = e^{kappa cos t} / (2 pi I0(kappa)). */
double or_vm_kernel(double kappa, double t)
{
    return exp(kappa * (cos(t) - 1.0)) / (OR_TWO_PI * or_i0e(kappa));
}

/* Ratios A_m(kappa) = I_m(kappa) / I_0(kappa), m = 0..M, which are the Fourier
 * coefficients of the von Mises kernel: K(t) = (1/2pi) sum_m A_m e^{i m t}.
 * From I_{m-1} - I_{m+1} = (2m/kappa) I_m the ratio r_m = I_m / I_{m-1} obeys
 * r_m = 1 / (2m/kappa + r_{m+1}); it is evaluated by downward recurrence from a
 * starting index far above M (a continued fraction), then A_m = r_1 ... r_m. */
void or_bessel_ratios(double kappa, int M, double *A)
{
    /* the tail of the continued fraction stops mattering once 2m/kappa >> 1 */
    int start = (M > (int)kappa ? M : (int)kappa) + 200 + (int)(10.0 * sqrt(kappa));
    double r = 0.0;
    double *rr = (double *)malloc(sizeof(double) * (size_t)(start + 2));
    for (int m = start; m >= 1; --m) {
        r = 1.0 / (2.0 * m / kappa + r);
        rr[m] = r;
    }
    A[0] = 1.0;
    for (int m = 1; m <= M; ++m) A[m] = A[m - 1] * rr[m];
    free(rr);
}

/* ------------------------------------------------------------------------ */
/* Eq. (kde) on the periodic grid: the plain KDE evaluated at the nodes.     */
/* rho_g = sum_i w_i * (2 pi / L) * K_{kappa_i}(theta_g - theta_i),          */
/* theta_g = 2 pi g / Ng.  Per-particle widths follow the adaptive estimator */
/* of Sec. II.C (each particle carries its own kernel).  With w_i = L/N the  */
/* mean density is 1.  kappa == NULL means the uniform width kappa_u; w ==   */
/* NULL means w_i = L/N.                                                     */
/* ------------------------------------------------------------------------ */
void or_deposit(const double *x, const double *kappa, double kappa_u, const double *w,
                int64_t N, int Ng, double L, double *rho)
{
    double *norm = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    for (int64_t i = 0; i < N; ++i) norm[i] = 1.0 / (OR_TWO_PI * or_i0e(kappa ? kappa[i] : kappa_u));
#pragma omp parallel for schedule(static)
    for (int g = 0; g < Ng; ++g) {
        double tg = OR_TWO_PI * (double)g / (double)Ng;
        double acc = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            double ti = OR_TWO_PI * x[i] / L;
            double k = kappa ? kappa[i] : kappa_u;
            double wi = w ? w[i] : L / (double)N;
            acc += wi * (OR_TWO_PI / L) * norm[i] * exp(k * (cos(tg - ti) - 1.0));
        }
        rho[g] = acc;
    }
    free(norm);
}

/* Field interpolation back to the particles through the same kernels:
 * E_i = sum_g (2 pi / Ng) K_{kappa_i}(theta_g - theta_i) E_g.  The weights are
 * those of the deposit divided by the cell length, so a constant field is
 * reproduced up to grid aliasing.  (The paper states only that E comes from
 * the Poisson solve; this is the reading used throughout.) */
void or_gather(const double *x, const double *kappa, double kappa_u, int64_t N,
               const double *E, int Ng, double L, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double ti = OR_TWO_PI * x[i] / L;
        double k = kappa ? kappa[i] : kappa_u;
        double nrm = 1.0 / (OR_TWO_PI * or_i0e(k));
        double acc = 0.0;
        for (int g = 0; g < Ng; ++g) {
            double tg = OR_TWO_PI * (double)g / (double)Ng;
            acc += (OR_TWO_PI / (double)Ng) * nrm * exp(k * (cos(tg - ti) - 1.0)) * E[g];
        }
        out[i] = acc;
    }
}

/* Poisson solve, spectral form: dE/dx = rho_total, E_m = rho_m / (i k_m),
 * k_m = 2 pi m / L, with the mean (m = 0) and, for even Ng, the Nyquist mode
 * set to zero.  Plain O(Ng^2) discrete Fourier transform. */
void or_poisson_spectral(const double *rho, int Ng, double L, double *E)
{
    double *re = (double *)calloc((size_t)Ng, sizeof(double));
    double *im = (double *)calloc((size_t)Ng, sizeof(double));
    for (int m = 0; m < Ng; ++m) {
        double sr = 0.0, si = 0.0;
        for (int j = 0; j < Ng; ++j) {
            double a = -OR_TWO_PI * (double)(((int64_t)m * j) % Ng) / (double)Ng;
            sr += rho[j] * cos(a);
            si += rho[j] * sin(a);
        }
        int ms = (2 * m < Ng) ? m : m - Ng; /* signed mode number */
        if (m == 0 || 2 * m == Ng) {
            re[m] = 0.0;
            im[m] = 0.0;
        } else {
            double k = OR_TWO_PI * (double)ms / L;
            /* (sr + i si) / (i k) = si / k - i sr / k */
            re[m] = si / k;
            im[m] = -sr / k;
        }
    }
    for (int j = 0; j < Ng; ++j) {
        double acc = 0.0;
        for (int m = 0; m < Ng; ++m) {
            double a = OR_TWO_PI * (double)(((int64_t)m * j) % Ng) / (double)Ng;
            acc += re[m] * cos(a) - im[m] * sin(a);
        }
        E[j] = acc / (double)Ng;
    }
    free(re);
    free(im);
}

/* Poisson solve, finite-difference form of Sec. III.A:
 * (phi_{j-1} - 2 phi_j + phi_{j+1}) / dx^2 = -rho_j,  E_j = (phi_{j-1} - phi_{j+1}) / (2 dx),
 * periodic.  The mean of rho is removed (the periodic Laplacian annihilates
 * constants), phi_0 = 0 fixes the gauge, and the remaining (Ng-1)-unknown
 * tridiagonal system is solved by the Thomas algorithm. */
void or_poisson_fd(const double *rho, int Ng, double L, double *E)
{
    double dx = L / (double)Ng, mean = 0.0;
    for (int j = 0; j < Ng; ++j) mean += rho[j];
    mean /= (double)Ng;
    double *phi = (double *)calloc((size_t)Ng, sizeof(double));
    int n = Ng - 1; /* unknowns phi_1..phi_{Ng-1}; rows j = 1..Ng-1 */
    if (n >= 1) {
        double *a = (double *)malloc(sizeof(double) * n), *b = (double *)malloc(sizeof(double) * n);
        double *c = (double *)malloc(sizeof(double) * n), *d = (double *)malloc(sizeof(double) * n);
        for (int r = 0; r < n; ++r) {
            a[r] = (r > 0) ? 1.0 : 0.0;      /* phi_{j-1} (phi_0 = 0 drops out) */
            c[r] = (r < n - 1) ? 1.0 : 0.0;  /* phi_{j+1} (phi_Ng = phi_0 = 0) */
            b[r] = -2.0;
            d[r] = -(rho[r + 1] - mean) * dx * dx;
        }
        for (int r = 1; r < n; ++r) {
            double f = a[r] / b[r - 1];
            b[r] -= f * c[r - 1];
            d[r] -= f * d[r - 1];
        }
        phi[n] = d[n - 1] / b[n - 1];
        for (int r = n - 2; r >= 0; --r) phi[r + 1] = (d[r] - c[r] * phi[r + 2]) / b[r];
        free(a); free(b); free(c); free(d);
    }
    for (int j = 0; j < Ng; ++j) {
        double pm = phi[(j - 1 + Ng) % Ng], pp = phi[(j + 1) % Ng];
        E[j] = (pm - pp) / (2.0 * dx);
    }
    free(phi);
}

/* Leap-frog push of Sec. III.A: v^{n+1/2} = v^{n-1/2} + kick * (q/m) E_i dt,
 * x^{n+1} = x^n + v^{n+1/2} dt, wrapped into [0, L).  kick = 1/2 on the first
 * step gives the usual half back-step start (v^{-1/2} = v^0 - (q/m) E^0 dt / 2). */
void or_push(double *x, double *v, const double *Ei, int64_t N, double L, double dt,
             double qm, double kick)
{
    for (int64_t i = 0; i < N; ++i) {
        v[i] += kick * qm * Ei[i] * dt;
        double xn = fmod(x[i] + v[i] * dt, L);
        if (xn < 0) xn += L;
        if (xn >= L) xn -= L;
        x[i] = xn;
    }
}

/* Field energy W = 1/2 sum_g E_g^2 dx (Sec. III.B, "energy of electric field"). */
double or_field_energy(const double *E, int Ng, double L)
{
    double s = 0.0;
    for (int g = 0; g < Ng; ++g) s += E[g] * E[g];
    return 0.5 * s * (L / (double)Ng);
}

/* ------------------------------------------------------------------------ */
/* Sec. II.B, Eq. (cv_def): leave-one-out cross-validation, dense pairs.     */
/* CV_theta = (1/n^2) sum_{i,j} Kbar_ij - (2/(n(n-1))) sum_i sum_{j!=i}      */
/*            K_{kappa_j}(theta_i - theta_j),                                */
/* with the two-fold convolution of two von Mises kernels in closed form:    */
/* Kbar_ij = I0(R_ij) / (2 pi I0(kappa_i) I0(kappa_j)),                      */
/* R_ij = sqrt(kappa_i^2 + kappa_j^2 + 2 kappa_i kappa_j cos(theta_i-theta_j))*/
/* (the integrand exp(k_i cos(t-t_i) + k_j cos(t-t_j)) = exp(R cos(t-phi))). */
/* Returns CV in x units ((2 pi / L) CV_theta).  Optionally returns the     */
/* per-particle leave-one-out density loo_i = (2pi/L) (1/(n-1))             */
/* sum_{j!=i} K_{kappa_j}(theta_i - theta_j) and the two terms separately.   */
/* kappa == NULL: uniform width kappa_u.                                     */
/* ------------------------------------------------------------------------ */
double or_cv_dense(const double *x, const double *kappa, double kappa_u, int64_t N, double L,
                   double *loo_out, double *int_f2_out, double *pair_mean_out)
{
    double *rowK = (double *)calloc((size_t)N, sizeof(double));
    double *rowKbar = (double *)calloc((size_t)N, sizeof(double));
    double *i0 = (double *)malloc(sizeof(double) * (size_t)N);
    for (int64_t i = 0; i < N; ++i) i0[i] = or_i0e(kappa ? kappa[i] : kappa_u);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < N; ++i) {
        double ti = OR_TWO_PI * x[i] / L, ki = kappa ? kappa[i] : kappa_u;
        double sK = 0.0, sKbar = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            double tj = OR_TWO_PI * x[j] / L, kj = kappa ? kappa[j] : kappa_u;
            double c = cos(ti - tj);
            double R = sqrt(fmax(ki * ki + kj * kj + 2.0 * ki * kj * c, 0.0));
            sKbar += or_i0e(R) * exp(R - ki - kj) / (OR_TWO_PI * i0[i] * i0[j]);
            if (j != i) sK += exp(kj * (c - 1.0)) / (OR_TWO_PI * i0[j]);
        }
        rowK[i] = sK;
        rowKbar[i] = sKbar;
    }
    double n = (double)N, sumK = 0.0, sumKbar = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        sumK += rowK[i];
        sumKbar += rowKbar[i];
        if (loo_out) loo_out[i] = (OR_TWO_PI / L) * rowK[i] / (n - 1.0);
    }
    double f2 = sumKbar / (n * n);
    double pm = sumK / (n * (n - 1.0));
    if (int_f2_out) *int_f2_out = (OR_TWO_PI / L) * f2;
    if (pair_mean_out) *pair_mean_out = (OR_TWO_PI / L) * pm;
    free(rowK); free(rowKbar); free(i0);
    return (OR_TWO_PI / L) * (f2 - 2.0 * pm);
}

/* Number of Fourier modes needed for the uniform-width spectral evaluation:
 * the smallest M with A_M(kappa) < 1e-18 (A_m decreases in m). */
int or_fourier_modes(double kappa)
{
    int M = 16;
    for (;;) {
        double *A = (double *)malloc(sizeof(double) * (size_t)(M + 1));
        or_bessel_ratios(kappa, M, A);
        int found = -1;
        for (int m = 1; m <= M; ++m)
            if (A[m] < 1e-18) { found = m; break; }
        free(A);
        if (found > 0) return found;
        M *= 2;
        if (M > (1 << 22)) return M;
    }
}

/* Eq. (cv_def) for a uniform width, evaluated exactly in Fourier space.
 * With S_m = sum_j e^{i m theta_j} and K = (1/2pi) sum_m A_m e^{imt}:
 *   sum_{i,j} K(theta_i - theta_j) = (1/2pi) sum_m A_m |S_m|^2,
 *   int fhat^2 dtheta              = (1/2pi) (1/n^2) sum_m A_m^2 |S_m|^2,
 *   n K(0)                         = (n/2pi) sum_m A_m,
 * sums over all integers m (terms m and -m are equal).  This is an identity,
 * not an approximation; the modes are cut where A_m < 1e-18.  S_m is built by
 * complex powers of e^{i theta_j}.  Optionally returns loo_i (x units). */
double or_cv_fourier(const double *x, int64_t N, double L, double kappa, double *loo_out,
                     double *int_f2_out, double *pair_mean_out)
{
    int M = or_fourier_modes(kappa);
    double *A = (double *)malloc(sizeof(double) * (size_t)(M + 1));
    or_bessel_ratios(kappa, M, A);
    double *Sr = (double *)calloc((size_t)(M + 1), sizeof(double));
    double *Si = (double *)calloc((size_t)(M + 1), sizeof(double));
    /* structure factor: accumulate per block of particles, then in block order */
    int64_t nblk = (N + 4095) / 4096;
    double *bSr = (double *)calloc((size_t)(nblk * (M + 1)), sizeof(double));
    double *bSi = (double *)calloc((size_t)(nblk * (M + 1)), sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < nblk; ++b) {
        double *pr = bSr + b * (M + 1), *pi = bSi + b * (M + 1);
        int64_t i1 = (b + 1) * 4096 < N ? (b + 1) * 4096 : N;
        for (int64_t j = b * 4096; j < i1; ++j) {
            double t = OR_TWO_PI * x[j] / L;
            double c1 = cos(t), s1 = sin(t), cr = 1.0, ci = 0.0;
            for (int m = 1; m <= M; ++m) {
                double nr = cr * c1 - ci * s1, ni = cr * s1 + ci * c1;
                cr = nr; ci = ni;
                if ((m & 63) == 0) { cr = cos(m * t); ci = sin(m * t); } /* re-anchor */
                pr[m] += cr;
                pi[m] += ci;
            }
        }
    }
    for (int64_t b = 0; b < nblk; ++b)
        for (int m = 1; m <= M; ++m) { Sr[m] += bSr[b * (M + 1) + m]; Si[m] += bSi[b * (M + 1) + m]; }
    free(bSr); free(bSi);
    double n = (double)N;
    double sumA = 1.0, sumAS2 = n * n, sumA2S2 = n * n; /* m = 0 terms */
    for (int m = 1; m <= M; ++m) {
        double s2 = Sr[m] * Sr[m] + Si[m] * Si[m];
        sumA += 2.0 * A[m];
        sumAS2 += 2.0 * A[m] * s2;
        sumA2S2 += 2.0 * A[m] * A[m] * s2;
    }
    double f2 = sumA2S2 / (OR_TWO_PI * n * n);
    double pairs = (sumAS2 - n * sumA) / OR_TWO_PI; /* sum_{i != j} K */
    double pm = pairs / (n * (n - 1.0));
    if (loo_out) {
        double K0 = sumA / OR_TWO_PI;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < N; ++i) {
            double t = OR_TWO_PI * x[i] / L;
            double c1 = cos(t), s1 = sin(t), cr = 1.0, ci = 0.0, acc = n;
            for (int m = 1; m <= M; ++m) {
                double nr = cr * c1 - ci * s1, ni = cr * s1 + ci * c1;
                cr = nr; ci = ni;
                if ((m & 63) == 0) { cr = cos(m * t); ci = sin(m * t); }
                /* Re(e^{i m t_i} conj(S_m)) */
                acc += 2.0 * A[m] * (cr * Sr[m] + ci * Si[m]);
            }
            loo_out[i] = (OR_TWO_PI / L) * (acc / OR_TWO_PI - K0) / (n - 1.0);
        }
    }
    if (int_f2_out) *int_f2_out = (OR_TWO_PI / L) * f2;
    if (pair_mean_out) *pair_mean_out = (OR_TWO_PI / L) * pm;
    free(A); free(Sr); free(Si);
    return (OR_TWO_PI / L) * (f2 - 2.0 * pm);
}

/* Appendix A: the CV function without leave-one-out,
 * (1/n^2) sum_{i,j} Kbar_ij - (2/n^2) sum_{i,j} K_ij (x units, uniform width). */
double or_cv_no_loo(const double *x, int64_t N, double L, double kappa)
{
    double f2, pm;
    or_cv_dense(x, NULL, kappa, N, L, NULL, &f2, &pm);
    double n = (double)N;
    double K0 = (OR_TWO_PI / L) / (OR_TWO_PI * or_i0e(kappa));
    /* sum_{i,j} K / n^2 = ((n-1)/n) * pair_mean + K0 / n */
    return f2 - 2.0 * (((n - 1.0) / n) * pm + K0 / n);
}

/* Sec. II.C: Silverman's particle-wise widths from the pilot estimate at the
 * CV-optimal width kappa_star.
 *   f~(X_i) = ((n-1) loo_i + K_{kappa*}(0)) / n    (pilot KDE at X_i, own kernel included)
 *   log g   = (1/n) sum_i log f~(X_i)
 *   lambda_i = (f~(X_i) / g)^(-alpha)
 *   h_i = h lambda_i with kappa = 1/h^2  =>  kappa_i = kappa* / lambda_i^2,
 * clamped to [kmin, kmax].  loo is in x units (as returned by the CV). */
void or_adapt_widths(const double *loo, int64_t N, double L, double kappa_star, double alpha,
                     double kmin, double kmax, double *kappa_out)
{
    double n = (double)N;
    double K0 = (OR_TWO_PI / L) / (OR_TWO_PI * or_i0e(kappa_star));
    double slog = 0.0;
    for (int64_t i = 0; i < N; ++i) slog += log(((n - 1.0) * loo[i] + K0) / n);
    double logg = slog / n;
    for (int64_t i = 0; i < N; ++i) {
        double f = ((n - 1.0) * loo[i] + K0) / n;
        double lam = exp(-alpha * (log(f) - logg));
        double k = kappa_star / (lam * lam);
        if (k < kmin) k = kmin;
        if (k > kmax) k = kmax;
        kappa_out[i] = k;
    }
}

/* Index of the smallest CV value; the smallest index wins an exact tie. */
int or_argmin(const double *cv, int n)
{
    int best = 0;
    for (int c = 1; c < n; ++c)
        if (cv[c] < cv[best]) best = c;
    return best;
}

/* ------------------------------------------------------------------------ */
/* Sec. III.A: electrostatic 1D periodic PIC cycle with KDE density.        */
/* Per step n (positions x^n, velocities v^{n-1/2}):                          */
/*   [width update every `width_every` steps: uniform-width CV over `cand`, */
/*    kappa* = argmin, Silverman widths from loo at kappa* (Sec. II.B-C)]    */
/*   rho_e = deposit; rho_total = background + charge * rho_e;               */
/*   E = Poisson(rho_total); W^n = field energy; E_i = gather;               */
/*   leap-frog push (half kick on step 0 when backstep != 0).                */
/* kappa: per-particle widths (in/out, used when per_particle != 0).         */
/* poisson_fd != 0 selects the finite-difference solve, else spectral.      */
/* cv_mode: 0 = dense pairs, 1 = Fourier form (uniform widths only).         */
/* W_out[nsteps], kstar_out[nsteps] (kappa* in force at each step) optional. */
/* ------------------------------------------------------------------------ */
int or_pic_run(double *x, double *v, double *kappa, int per_particle, double kappa_u, int64_t N,
               int Ng, double L, double dt, double qm, double charge, double background,
               int poisson_fd, int nsteps, int width_every, const double *cand, int n_cand,
               double alpha, double kmin, double kmax, int cv_mode, int backstep,
               double *W_out, double *kstar_out)
{
    double *rho = (double *)malloc(sizeof(double) * (size_t)Ng);
    double *E = (double *)malloc(sizeof(double) * (size_t)Ng);
    double *Ei = (double *)malloc(sizeof(double) * (size_t)N);
    double *loo = (double *)malloc(sizeof(double) * (size_t)N);
    double *cv = (double *)malloc(sizeof(double) * (size_t)(n_cand > 0 ? n_cand : 1));
    double kstar = kappa_u;
    for (int n = 0; n < nsteps; ++n) {
        if (width_every > 0 && n % width_every == 0 && n_cand > 0) {
            for (int c = 0; c < n_cand; ++c)
                cv[c] = cv_mode ? or_cv_fourier(x, N, L, cand[c], NULL, NULL, NULL)
                                : or_cv_dense(x, NULL, cand[c], N, L, NULL, NULL, NULL);
            kstar = cand[or_argmin(cv, n_cand)];
            if (per_particle) {
                if (cv_mode) or_cv_fourier(x, N, L, kstar, loo, NULL, NULL);
                else or_cv_dense(x, NULL, kstar, N, L, loo, NULL, NULL);
                or_adapt_widths(loo, N, L, kstar, alpha, kmin, kmax, kappa);
            } else {
                kappa_u = kstar;
            }
        }
        or_deposit(x, per_particle ? kappa : NULL, kappa_u, NULL, N, Ng, L, rho);
        for (int g = 0; g < Ng; ++g) rho[g] = background + charge * rho[g];
        if (poisson_fd) or_poisson_fd(rho, Ng, L, E);
        else or_poisson_spectral(rho, Ng, L, E);
        if (W_out) W_out[n] = or_field_energy(E, Ng, L);
        if (kstar_out) kstar_out[n] = kstar;
        or_gather(x, per_particle ? kappa : NULL, kappa_u, N, E, Ng, L, Ei);
        or_push(x, v, Ei, N, L, dt, qm, (n == 0 && backstep) ? 0.5 : 1.0);
    }
    free(rho); free(E); free(Ei); free(loo); free(cv);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. II.D: Anderson-Darling test of the positions against the uniform     */
/* distribution on the domain.  F[i] = F(X_i) are the values of the uniform */
/* CDF at the samples, in (0, 1).  With F_(1) <= ... <= F_(n) sorted:         */
/*   A^2 = -n - (1/n) sum_{i=1}^{n} (2i - 1) [ln F_(i) + ln(1 - F_(n+1-i))]   */
/* (Anderson & Darling 1954).  The sort is a library qsort; the sum runs in  */
/* index order.                                                              */
/* ------------------------------------------------------------------------ */
static int or_cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

double or_ad_statistic(const double *F, int64_t n)
{
    double *s = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    memcpy(s, F, sizeof(double) * (size_t)n);
    qsort(s, (size_t)n, sizeof(double), or_cmp_double);
    double sum = 0.0;
    for (int64_t i = 1; i <= n; ++i) sum += (2.0 * i - 1.0) * (log(s[i - 1]) + log(1.0 - s[n - i]));
    free(s);
    return -(double)n - sum / (double)n;
}

/* The uniform CDF at a position as the test sees it: at the resolution of the */
/* 32-bit position code, at the centre of the code's cell,                     */
/* F = (floor(x / L * 2^32) + 1/2) / 2^32, which lies strictly inside (0, 1).  */
double or_ad_cdf_of_position(double x, double L)
{
    double q = floor(x / L * 4294967296.0);
    if (q < 0.0) q = 0.0;
    if (q > 4294967295.0) q = 4294967295.0;
    return (q + 0.5) / 4294967296.0;
}

/* P(A^2 <= z) for n samples from the hypothesised distribution, following   */
/* Marsaglia & Marsaglia, "Evaluating the Anderson-Darling distribution",     */
/* J. Stat. Softw. 9(2), 2004: the limiting distribution by their two fitted  */
/* expressions (below and above z = 2), plus their finite-n correction, which */
/* is a function of n and of the limiting value.                             */
static double or_ad_limit(double z)
{
    if (z <= 0.0) return 0.0;
    if (z < 2.0)
        return exp(-1.2337141 / z) / sqrt(z) *
               (2.00012 + (0.247105 - (0.0649821 - (0.0347962 - (0.011672 - 0.00168691 * z) * z) * z) * z) * z);
    return exp(-exp(1.0776 - (2.30695 - (0.43424 - (0.082433 - (0.008056 - 0.0003146 * z) * z) * z) * z) * z));
}

static double or_ad_finite_n(int64_t n_, double x)
{
    const double n = (double)n_;
    if (x > 0.8)
        return (-130.2137 + (745.2337 - (1705.091 - (1950.646 - (1116.360 - 255.7844 * x) * x) * x) * x) * x) / n;
    const double c = 0.01265 + 0.1757 / n;
    if (x < c) {
        double t = x / c;
        t = sqrt(t) * (1.0 - t) * (49.0 * t - 102.0);
        return t * (0.0037 / (n * n) + 0.00078 / n + 0.00006) / n;
    }
    double t = (x - c) / (0.8 - c);
    t = -0.00022633 + (6.54034 - (14.6538 - (14.458 - (8.259 - 1.91864 * t) * t) * t) * t) * t;
    return t * (0.04213 + 0.01365 / n) / n;
}

double or_ad_cdf(double z, int64_t n)
{
    const double x = or_ad_limit(z);
    double p = x + or_ad_finite_n(n, x);
    if (p < 0.0) p = 0.0;
    if (p > 1.0) p = 1.0;
    return p;
}

/* Natural log of the p-value of the test: the probability, under the uniform */
/* hypothesis, of an A^2 at least this large.  Up to A^2 = 7 it is           */
/* 1 - P(A^2 <= z) from the expressions above.  Beyond, where those fitted    */
/* expressions stop resolving the tail (they reach 1 to double precision), it */
/* follows the large-z behaviour of the limiting distribution: A^2 is a sum   */
/* of chi^2_1 variables weighted 1/(j(j+1)); the j = 1 term dominates the     */
/* tail, so P(A^2 > z) ~ C z^{-1/2} e^{-z}.  The constant is taken from the   */
/* value at z = 7, so the p-value is continuous and keeps decreasing, and the */
/* log form does not underflow for the huge statistics of strongly clustered  */
/* samples.                                                                   */
#define OR_AD_ZJOIN 7.0
double or_ad_log_pvalue(double a2, int64_t n)
{
    if (a2 <= OR_AD_ZJOIN) return log(1.0 - or_ad_cdf(a2, n));
    return log(1.0 - or_ad_cdf(OR_AD_ZJOIN, n)) + 0.5 * log(OR_AD_ZJOIN / a2) + (OR_AD_ZJOIN - a2);
}

double or_ad_pvalue(double a2, int64_t n) { return exp(or_ad_log_pvalue(a2, n)); }

/* Sec. II.D update rule for one step, written on logs of p-values.  State:  */
/* lp_th = ln p_th (a value >= 0 means "no step yet": it starts at            */
/* ln(2 threshold)).  Returns 1 when the width is to be re-optimised at this  */
/* step (the caller then minimises CV and takes the new target), else 0:     */
/*   p > 2 threshold            -> p_th = 2 threshold                         */
/*   else if p < p_th / 2       -> optimise, p_th = p                         */
int or_ad_schedule_step(double lp, double threshold, double *lp_th)
{
    const double l2t = log(2.0 * threshold);
    if (*lp_th >= 0.0) *lp_th = l2t;
    if (lp > l2t) {
        *lp_th = l2t;
        return 0;
    }
    if (lp < *lp_th - log(2.0)) {
        *lp_th = lp;
        return 1;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. III.A PIC cycle with the width-update algorithm of Sec. II.D on a    */
/* uniform width.  Every step, before the deposit: the AD p-value of the      */
/* positions, the update rule above; on an optimisation step the uniform CV   */
/* over `cand` (Fourier form) gives the target width.  Widths are smoothed in */
/* h = kappa^{-1/2}: h = rate h_target + (1 - rate) h.  Until the first       */
/* optimisation the caller's width kappa_u is used; the first optimisation    */
/* sets h = h_target (there is no earlier optimum to smooth from).           */
/* State (in/out): *lp_th (>= 0 on entry = start), *h_target (0 = no          */
/* optimisation yet), *kappa_u.  Outputs per step (optional): W_out,          */
/* kappa_out (width in force), lp_out (ln p-value), cv_out (1 on optimisation)*/
/* ------------------------------------------------------------------------ */
int or_pic_run_ad(double *x, double *v, double *kappa_u, int64_t N, int Ng, double L, double dt, double qm,
                  double charge, double background, int poisson_fd, int nsteps, const double *cand, int n_cand,
                  double threshold, double rate, int backstep, int64_t step0, double *lp_th, double *h_target,
                  double *W_out, double *kappa_out, double *lp_out, int *cv_out)
{
    double *rho = (double *)malloc(sizeof(double) * (size_t)Ng);
    double *E = (double *)malloc(sizeof(double) * (size_t)Ng);
    double *Ei = (double *)malloc(sizeof(double) * (size_t)N);
    double *F = (double *)malloc(sizeof(double) * (size_t)N);
    double *cv = (double *)malloc(sizeof(double) * (size_t)(n_cand > 0 ? n_cand : 1));
    double h = 1.0 / sqrt(*kappa_u);
    for (int n = 0; n < nsteps; ++n) {
        for (int64_t i = 0; i < N; ++i) F[i] = or_ad_cdf_of_position(x[i], L);
        const double lp = or_ad_log_pvalue(or_ad_statistic(F, N), N);
        const int opt = or_ad_schedule_step(lp, threshold, lp_th);
        if (opt) {
            for (int c = 0; c < n_cand; ++c) cv[c] = or_cv_fourier(x, N, L, cand[c], NULL, NULL, NULL);
            const double ht = 1.0 / sqrt(cand[or_argmin(cv, n_cand)]);
            if (!(*h_target > 0.0)) h = ht;
            *h_target = ht;
        }
        if (*h_target > 0.0) h = rate * *h_target + (1.0 - rate) * h;
        *kappa_u = 1.0 / (h * h);
        if (lp_out) lp_out[n] = lp;
        if (cv_out) cv_out[n] = opt;
        if (kappa_out) kappa_out[n] = *kappa_u;
        or_deposit(x, NULL, *kappa_u, NULL, N, Ng, L, rho);
        for (int g = 0; g < Ng; ++g) rho[g] = background + charge * rho[g];
        if (poisson_fd) or_poisson_fd(rho, Ng, L, E);
        else or_poisson_spectral(rho, Ng, L, E);
        if (W_out) W_out[n] = or_field_energy(E, Ng, L);
        or_gather(x, NULL, *kappa_u, N, E, Ng, L, Ei);
        or_push(x, v, Ei, N, L, dt, qm, (step0 + n == 0 && backstep) ? 0.5 : 1.0);
    }
    free(rho); free(E); free(Ei); free(F); free(cv);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Standard-PIC shapes for the comparison of Sec. IV (Fig. compare_high_order):*/
/* the centred cardinal B-spline of degree p, B_p(t) = N_{p+1}(t + (p+1)/2),  */
/* with the uniform B-spline of order m on the knots 0..m given by the         */
/* Cox-de Boor recursion N_1 = 1 on [0, 1),                                    */
/* N_m(x) = (x N_{m-1}(x) + (m - x) N_{m-1}(x - 1)) / (m - 1).                */
/* A shape of width h is S(x) = (1/h) B_p(x/h), support (p + 1) h; h = dx is   */
/* the standard PIC shape ("width (order + 1) dx").                            */
/* ------------------------------------------------------------------------ */
static double or_nspline(int m, double x)
{
    if (x < 0.0 || x >= (double)m) return 0.0;
    if (m == 1) return 1.0;
    return (x * or_nspline(m - 1, x) + ((double)m - x) * or_nspline(m - 1, x - 1.0)) / (double)(m - 1);
}

double or_bspline(int p, double t) { return or_nspline(p + 1, t + 0.5 * (double)(p + 1)); }

/* shortest periodic signed separation a - b on a circle of length L */
static double or_periodic(double a, double b, double L)
{
    double d = fmod(a - b, L);
    if (d >= 0.5 * L) d -= L;
    if (d < -0.5 * L) d += L;
    return d;
}

/* deposit with the shape at the nodes: rho_g = sum_i w_i S(x_g - x_i), w_i = L/N, */
/* periodic ((p + 1) h < L keeps one image in reach)                               */
void or_deposit_bspline(const double *x, int64_t N, int p, double h, int Ng, double L, double *rho)
{
#pragma omp parallel for schedule(static)
    for (int g = 0; g < Ng; ++g) {
        const double xg = L * (double)g / (double)Ng;
        double acc = 0.0;
        for (int64_t i = 0; i < N; ++i) acc += (L / (double)N) / h * or_bspline(p, or_periodic(xg, x[i], L) / h);
        rho[g] = acc;
    }
}

/* field interpolation with the same shape: E_i = sum_g E_g (dx / h) B_p((x_g - x_i)/h) */
void or_gather_bspline(const double *x, int64_t N, int p, double h, const double *E, int Ng, double L, double *out)
{
    const double dx = L / (double)Ng;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double acc = 0.0;
        for (int g = 0; g < Ng; ++g)
            acc += E[g] * (dx / h) * or_bspline(p, or_periodic(L * (double)g / (double)Ng, x[i], L) / h);
        out[i] = acc;
    }
}

/* Eq. (cv_def) for the first-order (CIC) shape of width h, in x units:          */
/* int fhat^2 = (1/n^2) sum_{i,j} (S * S)(x_i - x_j) with S * S = (1/h) B_3(./h)   */
/* (the convolution of two degree-1 B-splines is the cubic one), minus          */
/* 2/(n(n-1)) sum_{i != j} S(x_i - x_j).  Dense over all pairs; 2h < L/2.         */
double or_cv_cic(const double *x, int64_t N, double L, double h)
{
    double *row3 = (double *)malloc(sizeof(double) * (size_t)N);
    double *row1 = (double *)malloc(sizeof(double) * (size_t)N);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < N; ++i) {
        double a3 = 0.0, a1 = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            const double t = or_periodic(x[i], x[j], L) / h;
            a3 += or_bspline(3, t) / h;
            if (j != i) a1 += or_bspline(1, t) / h;
        }
        row3[i] = a3;
        row1[i] = a1;
    }
    double s3 = 0.0, s1 = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        s3 += row3[i];
        s1 += row1[i];
    }
    free(row3);
    free(row1);
    const double n = (double)N;
    return s3 / (n * n) - 2.0 * s1 / (n * (n - 1.0));
}

/* Standard PIC cycle (the baseline of Sec. III.B's ensemble comparison): the  */
/* step of or_pic_run with the B-spline shape of degree p and width h in place  */
/* of the von Mises kernel, spectral Poisson, the same leap-frog push.           */
int or_pic_run_bspline(double *x, double *v, int64_t N, int p, double h, int Ng, double L, double dt, double qm,
                       double charge, double background, int nsteps, int backstep, double *W_out)
{
    double *rho = (double *)malloc(sizeof(double) * (size_t)Ng);
    double *E = (double *)malloc(sizeof(double) * (size_t)Ng);
    double *Ei = (double *)malloc(sizeof(double) * (size_t)N);
    for (int n = 0; n < nsteps; ++n) {
        or_deposit_bspline(x, N, p, h, Ng, L, rho);
        for (int g = 0; g < Ng; ++g) rho[g] = background + charge * rho[g];
        or_poisson_spectral(rho, Ng, L, E);
        if (W_out) W_out[n] = or_field_energy(E, Ng, L);
        or_gather_bspline(x, N, p, h, E, Ng, L, Ei);
        or_push(x, v, Ei, N, L, dt, qm, (n == 0 && backstep) ? 0.5 : 1.0);
    }
    free(rho); free(E); free(Ei);
    return 0;
}

/* Sec. III.B: damping rate from the field energy.  The slope of ln W through
 * the first two strict local maxima after t = 0 (steps n >= 1) is the energy
 * decay rate; the amplitude rate gamma is half of it.  Returns 0 and sets
 * *gamma, or -1 if fewer than two maxima exist. */
int or_damping_rate(const double *W, int n, double dt, double *gamma, int *p1, int *p2)
{
    int found = 0, idx[2] = {0, 0};
    for (int k = 1; k + 1 < n && found < 2; ++k)
        if (W[k] > W[k - 1] && W[k] > W[k + 1]) idx[found++] = k;
    if (found < 2) return -1;
    *gamma = 0.5 * (log(W[idx[1]]) - log(W[idx[0]])) / ((idx[1] - idx[0]) * dt);
    if (p1) *p1 = idx[0];
    if (p2) *p2 = idx[1];
    return 0;
}

/* Eq. (kde) at arbitrary points: value of the deposit's density (x units) at
 * positions xp[p] -- the same definition as or_deposit, one output at a time,
 * for sampled checks of large problems. */
void or_kde_at(const double *x, const double *kappa, double kappa_u, const double *w, int64_t N, double L,
               const double *xp, int64_t np, double *out)
{
    double *norm = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    for (int64_t i = 0; i < N; ++i) norm[i] = 1.0 / (OR_TWO_PI * or_i0e(kappa ? kappa[i] : kappa_u));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t p = 0; p < np; ++p) {
        double tp = OR_TWO_PI * xp[p] / L, acc = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            double ti = OR_TWO_PI * x[i] / L;
            double k = kappa ? kappa[i] : kappa_u;
            double wi = w ? w[i] : L / (double)N;
            acc += wi * (OR_TWO_PI / L) * norm[i] * exp(k * (cos(tp - ti) - 1.0));
        }
        out[p] = acc;
    }
    free(norm);
}
