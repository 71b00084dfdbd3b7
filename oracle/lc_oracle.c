/*
 * lc_oracle.c -- plain FP64 CPU oracle for the light-cone (retarded) radiation
 * field of Ahn 2015, "Light-Cone Effect of Radiation Fields in Cosmological
 * Radiative Transfer Simulations".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or helper with
 * the CUDA implementation.
 *
 * What it computes (by definition, slowly, in double precision):
 *
 *   J(i) = U * sum_n sum_{i'} G_n(i - i') f_n(i')                (Eq. 11, 9)
 *
 * i.e. the periodic real-space convolution of the gridded source term of
 * every past slice n with that slice's effective retarded Green's function
 * G_n (Eq. 10), summed over slices (algorithm step 6 of Section 2.2).  No FFT
 * is used: the oracle is the direct sum of Eq. 11.
 *
 * G_n(d) for a cell displacement d is the average over s^3 sub-cell samples
 * of the radial kernel (the LW one of Eq. 17, or the exponentially attenuated
 * one of lco_fk) summed over all periodic images of a unit source
 * that fall in the slice's spherical shell (Eq. 10 and step 2 of Section
 * 2.2), then scaled so that l^3 * sum_d G_n(d) equals the analytic shell
 * integral of 4 pi r^2 g(r).  The readings of the paper that this needs
 * (half-open shells, exact integer shell classification, the observing time
 * of a step, the sub-sampling, the normalisation, units) are stated beside
 * the code that takes them.
 *
 * Cosmology: flat LCDM without radiation, H(z) = 100 h sqrt(Om (1+z)^3 + 1 - Om)
 * km/s/Mpc; conformal distance chi(z1, z2) = int_{z1}^{z2} c dz / H(z) in
 * comoving Mpc (Eq. 6: the null geodesic has d|x|/dtau = 1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_C_KMS 299792.458
#define OR_PI 3.14159265358979323846
#define OR_MPC_KM 3.0856775814913673e19
#define OR_MYR_S 3.15576e13

/* ------------------------------------------------------------------ */
/* Gauss-Legendre 20-point rule, nodes by Newton iteration on P_20.    */
/* ------------------------------------------------------------------ */
#define OR_GL_N 20
static double gl_x[OR_GL_N], gl_w[OR_GL_N];

__attribute__((constructor)) static void gl_init(void) {
    const int n = OR_GL_N;
    for (int i = 0; i < n; ++i) {
        double x = cos(OR_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 1; k < n; ++k) {
                double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
                p0 = p1;
                p1 = p2;
            }
            /* p1 = P_n(x), p0 = P_{n-1}(x) */
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        gl_x[i] = x;
        gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

/* ------------------------------------------------------------------ */
/* Cosmology (Eqs. 5-6)                                                */
/* ------------------------------------------------------------------ */
double lco_hubble(double om, double h, double z) {
    double a = 1.0 + z;
    return 100.0 * h * sqrt(om * a * a * a + (1.0 - om));
}

/* chi(z1, z2) = int_{z1}^{z2} c / H(z) dz [comoving Mpc]; composite 20-point
 * Gauss-Legendre on panels no wider than 0.05 in z. */
double lco_chi(double om, double h, double z1, double z2) {
    if (z1 == z2) return 0.0;
    double sgn = 1.0;
    if (z2 < z1) {
        double t = z1;
        z1 = z2;
        z2 = t;
        sgn = -1.0;
    }
    int np = (int)ceil((z2 - z1) / 0.05);
    if (np < 1) np = 1;
    double w = (z2 - z1) / np, sum = 0.0;
    for (int p = 0; p < np; ++p) {
        double mid = z1 + (p + 0.5) * w, half = 0.5 * w, ps = 0.0;
        for (int i = 0; i < OR_GL_N; ++i) ps += gl_w[i] * OR_C_KMS / lco_hubble(om, h, mid + half * gl_x[i]);
        sum += half * ps;
    }
    return sgn * sum;
}

/* Cosmic time since the big bang [Myr], flat LCDM closed form
 * t = 2 / (3 H0 sqrt(OL)) asinh( sqrt(OL/Om) (1+z)^{-3/2} );  Om = 1 gives
 * t = 2 / (3 H0) (1+z)^{-3/2}. */
double lco_time_myr(double om, double h, double z) {
    double H0 = 100.0 * h;                      /* km/s/Mpc */
    double tH = OR_MPC_KM / H0 / OR_MYR_S;      /* 1/H0 in Myr */
    double ol = 1.0 - om;
    double y = pow(1.0 + z, -1.5);
    if (ol <= 0.0) return 2.0 / 3.0 * tH * y;
    return 2.0 / (3.0 * sqrt(ol)) * tH * asinh(sqrt(ol / om) * y);
}

double lco_z_of_time(double om, double h, double t_myr) {
    double H0 = 100.0 * h;
    double tH = OR_MPC_KM / H0 / OR_MYR_S;
    double ol = 1.0 - om;
    double y;
    if (ol <= 0.0) y = 1.5 * t_myr / tH;
    else y = sinh(1.5 * sqrt(ol) * t_myr / tH) * sqrt(om / ol);
    return pow(y, -2.0 / 3.0) - 1.0;
}

/* Source redshift z_s seen at comoving distance r by an observer at z_obs:
 * chi(z_obs, z_s) = r.  Safeguarded Newton (d chi / dz = c / H) inside a
 * bisection bracket. */
double lco_zs_of_r(double om, double h, double z_obs, double r) {
    if (r <= 0.0) return z_obs;
    double lo = z_obs, hi = z_obs + 1.0;
    while (lco_chi(om, h, z_obs, hi) < r) {
        lo = hi;
        hi = z_obs + 2.0 * (hi - z_obs);
        if (hi > 1e8) return hi;
    }
    double z = 0.5 * (lo + hi);
    for (int it = 0; it < 200; ++it) {
        double f = lco_chi(om, h, z_obs, z) - r;
        if (f > 0.0) hi = z;
        else lo = z;
        double zn = z - f * lco_hubble(om, h, z) / OR_C_KMS;
        if (!(zn > lo && zn < hi)) zn = 0.5 * (lo + hi);
        if (fabs(zn - z) <= 1e-15 * (1.0 + z)) {
            z = zn;
            break;
        }
        z = zn;
    }
    return z;
}

/* Eq. 16 */
double lco_alpha(double om, double h, double zs) {
    return pow(h / 0.7, -1.0) * pow(om / 0.27, -0.5) * pow((1.0 + zs) / 21.0, -0.5);
}

/* Eq. 15: LW modulation with its hard horizon at r / alpha = 97.39. */
double lco_fmod(double r, double alpha) {
    if (r / alpha > 97.39) return 0.0;
    return 1.7 * exp(-pow(r / (116.29 * alpha), 0.68)) - 0.7;
}

/* The rough LW horizon of Section 1, 100 [21 / (1 + z)]^0.5 comoving Mpc,
 * read with z the emission redshift z_s (as Eq. 16 reads alpha). */
double lco_rough_horizon(double zs) { return 100.0 * sqrt(21.0 / (1.0 + zs)); }

/* Radial kernels.  The generic RGF (Eq. 7) carries a dilution factor that
 * this method needs only as a function of distance.  Kernel kind kk:
 *   0: Lyman-Werner, Eq. 14 / Eq. 17 with f_mod of Eq. 15 at alpha(z_s);
 *   1: the same (1+z)^3 / ((4 pi)^2 (1+z_s) r^2) dilution with f_mod replaced
 *      by exp(-r / kl) for r < kr and 0 beyond (kl: attenuation length,
 *      kr: cut-off, comoving Mpc);
 *   2: Lyman-Werner with the rough horizon of Section 1 in place of Eq. 15's
 *      97.39 alpha: the modulation of Eq. 15 without its cut, clamped at 0
 *      (it turns negative at r / alpha = 116.29 ln(1.7/0.7)^(1/0.68)), for
 *      r <= 100 [21 / (1 + z_s)]^0.5, and 0 beyond.
 * lco_fk is the factor that multiplies the dilution. */
double lco_fk(int kk, double kl, double kr, double om, double h, double zs, double r) {
    if (kk == 1) return r < kr ? exp(-r / kl) : 0.0;
    if (kk == 2) {
        if (r > lco_rough_horizon(zs)) return 0.0;
        double f = 1.7 * exp(-pow(r / (116.29 * lco_alpha(om, h, zs)), 0.68)) - 0.7;
        return f > 0.0 ? f : 0.0;
    }
    return lco_fmod(r, lco_alpha(om, h, zs));
}

/* field per unit source luminosity at comoving distance r (light cone: z_s
 * from chi(z_obs, z_s) = r).  Units: luminosity / Mpc^2 / sr. */
double lco_gk(int kk, double kl, double kr, double om, double h, double z_obs, double r) {
    double zs = lco_zs_of_r(om, h, z_obs, r);
    double fm = lco_fk(kk, kl, kr, om, h, zs, r);
    if (fm == 0.0) return 0.0;
    double zo = 1.0 + z_obs;
    return zo * zo * zo * fm / ((4.0 * OR_PI) * (4.0 * OR_PI) * (1.0 + zs) * r * r);
}

/* Eq. 17 with Eq. 14: the LW kernel. */
double lco_g(double om, double h, double z_obs, double r) { return lco_gk(0, 0.0, 0.0, om, h, z_obs, r); }

double lco_horizon(double om, double h, double z_obs);
double lco_rough_horizon_r(double om, double h, double z_obs);
/* the kernel's horizon: LW below; the cut-off for kind 1; the rough one for kind 2 */
double lco_horizonk(int kk, double kl, double kr, double om, double h, double z_obs) {
    (void)kl;
    if (kk == 1) return kr;
    if (kk == 2) return lco_rough_horizon_r(om, h, z_obs);
    return lco_horizon(om, h, z_obs);
}

/* The radius where r = 100 [21 / (1 + z_s(r))]^0.5 (kernel kind 2).  The
 * right-hand side falls as r grows, so the root is unique.  Bisection. */
double lco_rough_horizon_r(double om, double h, double z_obs) {
    double lo = 0.0, hi = lco_rough_horizon(z_obs);
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        double phi = mid - lco_rough_horizon(lco_zs_of_r(om, h, z_obs, mid));
        if (phi > 0.0) hi = mid;
        else lo = mid;
        if (hi - lo <= 1e-14 * hi) break;
    }
    return 0.5 * (lo + hi);
}

/* LW horizon r_h: the radius where r / alpha(z_s(r)) = 97.39 (Eq. 15, with
 * z = z_s per Section 1 and Eq. 16).  Bisection. */
double lco_horizon(double om, double h, double z_obs) {
    double lo = 0.0, hi = 97.39 * lco_alpha(om, h, z_obs);
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        double phi = mid - 97.39 * lco_alpha(om, h, lco_zs_of_r(om, h, z_obs, mid));
        if (phi > 0.0) hi = mid;
        else lo = mid;
        if (hi - lo <= 1e-14 * hi) break;
    }
    return 0.5 * (lo + hi);
}

/* integrand of the shell integral: 4 pi r^2 g(r) */
static double shell_integrand(int kk, double kl, double kr, double om, double h, double z_obs, double r) {
    double zs = lco_zs_of_r(om, h, z_obs, r);
    double fm = lco_fk(kk, kl, kr, om, h, zs, r);
    double zo = 1.0 + z_obs;
    return zo * zo * zo * fm / (4.0 * OR_PI * (1.0 + zs));
}

static double gl_panel(int kk, double kl, double kr, double om, double h, double z_obs, double a, double b) {
    double mid = 0.5 * (a + b), half = 0.5 * (b - a), s = 0.0;
    for (int i = 0; i < OR_GL_N; ++i)
        s += gl_w[i] * shell_integrand(kk, kl, kr, om, h, z_obs, mid + half * gl_x[i]);
    return half * s;
}

/* Kernel kind 2: the radius where the unclamped modulation of Eq. 15 reaches
 * 0, r = 116.29 ln(1.7 / 0.7)^(1 / 0.68) alpha(z_s(r)); the clamped kernel is
 * 0 beyond it.  Bisection (alpha falls with r, so the root is unique). */
double lco_fzero_r(double om, double h, double z_obs) {
    const double x0 = 116.29 * pow(log(1.7 / 0.7), 1.0 / 0.68);
    double lo = 0.0, hi = x0 * lco_alpha(om, h, z_obs);
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        double phi = mid - x0 * lco_alpha(om, h, lco_zs_of_r(om, h, z_obs, mid));
        if (phi > 0.0) hi = mid;
        else lo = mid;
        if (hi - lo <= 1e-14 * hi) break;
    }
    return 0.5 * (lo + hi);
}

/* I = int_{r_lo}^{min(r_hi, r_h)} 4 pi r^2 g(r) dr.  Panels are graded
 * geometrically towards r = 0 because f_mod carries r^0.68.  For kernel kind
 * 2 the upper limit also stops where the clamped modulation reaches 0, so
 * that no panel straddles the kink of the clamp. */
double lco_shell_integralk(int kk, double kl, double kr, double om, double h, double z_obs, double r_lo,
                           double r_hi) {
    double rh = lco_horizonk(kk, kl, kr, om, h, z_obs);
    double b = r_hi < rh ? r_hi : rh;
    if (kk == 2) {
        double rz = lco_fzero_r(om, h, z_obs);
        if (rz < b) b = rz;
    }
    if (!(r_lo < b)) return 0.0;
    double sum = 0.0;
    if (r_lo <= 0.0) {
        for (int k = 0; k < 60; ++k) sum += gl_panel(kk, kl, kr, om, h, z_obs, ldexp(b, -(k + 1)), ldexp(b, -k));
        return sum;
    }
    double x = r_lo;
    while (x < b) {
        double w = 0.5 * x;
        if (w > 1.0) w = 1.0;
        if (x + w > b) w = b - x;
        sum += gl_panel(kk, kl, kr, om, h, z_obs, x, x + w);
        x += w;
    }
    return sum;
}

double lco_shell_integral(double om, double h, double z_obs, double r_lo, double r_hi) {
    return lco_shell_integralk(0, 0.0, 0.0, om, h, z_obs, r_lo, r_hi);
}

/* ------------------------------------------------------------------ */
/* Step edges                                                          */
/* ------------------------------------------------------------------ */
/* kind 0: explicit copy; 1: equal cosmic time z_start -> z_end; 2: equal
 * conformal time ending at z_end with width r_h(z_end) / n_shell. */
int lco_step_edgesk(int kk, double kl, double kr, double om, double h, int kind, int n_steps, double z_start,
                    double z_end, int n_shell, const double* z_explicit, double* out) {
    if (n_steps < 1) return 1;
    if (kind == 0) {
        for (int k = 0; k <= n_steps; ++k) out[k] = z_explicit[k];
        return 0;
    }
    if (kind == 1) {
        double t0 = lco_time_myr(om, h, z_start), t1 = lco_time_myr(om, h, z_end);
        for (int k = 0; k <= n_steps; ++k) out[k] = lco_z_of_time(om, h, t0 + (t1 - t0) * k / n_steps);
        out[0] = z_start;
        out[n_steps] = z_end;
        return 0;
    }
    if (kind == 2) {
        if (n_shell < 1) return 1;
        double dtau = lco_horizonk(kk, kl, kr, om, h, z_end) / n_shell;
        for (int k = 0; k < n_steps; ++k) out[k] = lco_zs_of_r(om, h, z_end, (n_steps - k) * dtau);
        out[n_steps] = z_end;
        return 0;
    }
    return 1;
}

int lco_step_edges(double om, double h, int kind, int n_steps, double z_start, double z_end, int n_shell,
                   const double* z_explicit, double* out) {
    return lco_step_edgesk(0, 0.0, 0.0, om, h, kind, n_steps, z_start, z_end, n_shell, z_explicit, out);
}

/* ------------------------------------------------------------------ */
/* Problem description                                                 */
/* ------------------------------------------------------------------ */
typedef struct {
    int n;               /* grid side N */
    double box;          /* L, comoving Mpc */
    double om, h;        /* cosmology */
    int n_steps;
    const double* z_edges; /* n_steps + 1 decreasing redshifts */
    int subsamples;      /* s, even */
    int normalise;       /* 1: scale G_n so that l^3 sum G_n = I_n */
    double out_unit;     /* U */
    int kernel;          /* radial kernel kind (see lco_fk) */
    double k_length, k_rmax;
    int n_shell_max;     /* > 0: at most this many slices per step (the newest ones) */
} lco_problem;

/* Active slices of observation step s.  Step s observes at tau_{s+1} (the end
 * of the step, so sources pushed at step s are included).  Slice n = s - j
 * covers the shell [chi(z_{s+1}, z_{n+1}), chi(z_{s+1}, z_n)) (Eq. 9 with a
 * half-open window); it is active while its inner radius is below
 * r_h (1 - 1e-9), and, when n_shell_max > 0, while j < n_shell_max (the
 * number of lookback slices kept per observing time, which the paragraph
 * after the algorithm of Section 2.2 lets vary; here a user's cap). */
int lco_shells(const lco_problem* P, int s, double* r_lo, double* r_hi, double* r_h) {
    if (s < 0 || s >= P->n_steps) return -1;
    double zo = P->z_edges[s + 1];
    double rh = lco_horizonk(P->kernel, P->k_length, P->k_rmax, P->om, P->h, zo);
    if (r_h) *r_h = rh;
    int A = 0;
    for (int j = 0; j <= s; ++j) {
        if (P->n_shell_max > 0 && j >= P->n_shell_max) break;
        int n = s - j;
        double lo = lco_chi(P->om, P->h, zo, P->z_edges[n + 1]);
        double hi = lco_chi(P->om, P->h, zo, P->z_edges[n]);
        /* a slice whose inner radius reaches the horizon (to 1e-9 relative)
         * carries no weight and is dropped */
        if (!(lo < rh * (1.0 - 1e-9))) break;
        if (r_lo) r_lo[A] = lo;
        if (r_hi) r_hi[A] = hi;
        ++A;
    }
    return A;
}

/* Octant storage of the shell Green's functions of one step:
 * G[j * (M+1)^3 + (a*(M+1) + b)*(M+1) + c], folded displacement a, b, c in
 * [0, M], M = N / 2 (G is even along each axis and periodic). */
typedef struct {
    int A, M;
    double* G;
    double* I;   /* analytic shell integrals */
    double* sum; /* sum over the full grid of the un-normalised G_j */
} octant_set;

static void octant_free(octant_set* o) {
    free(o->G);
    free(o->I);
    free(o->sum);
    memset(o, 0, sizeof(*o));
}

/* ceil of x for a non-negative double, as int64 */
static int64_t ceil_i64(double x) { return (int64_t)ceil(x); }

static int build_octants(const lco_problem* P, int s, octant_set* out) {
    memset(out, 0, sizeof(*out));
    const int N = P->n, M = N / 2, S = P->subsamples;
    const double l = P->box / N;
    const double delta = l / (2.0 * S); /* sample radii r = delta * sqrt(R) */
    const double zo = P->z_edges[s + 1];
    double* rlo = (double*)malloc(sizeof(double) * (s + 1));
    double* rhi = (double*)malloc(sizeof(double) * (s + 1));
    double rh;
    int A = lco_shells(P, s, rlo, rhi, &rh);
    out->A = A;
    out->M = M;
    const size_t oct = (size_t)(M + 1) * (M + 1) * (M + 1);
    out->G = (double*)calloc((size_t)(A > 0 ? A : 1) * oct, sizeof(double));
    out->I = (double*)calloc(A > 0 ? A : 1, sizeof(double));
    out->sum = (double*)calloc(A > 0 ? A : 1, sizeof(double));
    if (A == 0) {
        free(rlo);
        free(rhi);
        return 0;
    }
    /* Integer shell boundaries in units of delta^2: sample with integer
     * squared radius R lies in shell j iff bnd[j] <= R < bnd[j+1]
     * (r_lo <= r < r_hi exactly), and inside the horizon iff R <= Rh. */
    int64_t* bnd = (int64_t*)malloc(sizeof(int64_t) * (A + 1));
    bnd[0] = ceil_i64((rlo[0] / delta) * (rlo[0] / delta));
    for (int j = 0; j < A; ++j) bnd[j + 1] = ceil_i64((rhi[j] / delta) * (rhi[j] / delta));
    int64_t Rh = (int64_t)floor((rh / delta) * (rh / delta));
    /* g at every admissible R (a sum of three odd squares, R = 3 mod 8). */
    int64_t ntab = Rh >= 3 ? (Rh - 3) / 8 + 1 : 0;
    double* tab = (double*)malloc(sizeof(double) * (ntab > 0 ? ntab : 1));
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t t = 0; t < ntab; ++t) {
        double r = delta * sqrt((double)(8 * t + 3));
        tab[t] = lco_gk(P->kernel, P->k_length, P->k_rmax, P->om, P->h, zo, r);
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < A; ++j)
        out->I[j] = lco_shell_integralk(P->kernel, P->k_length, P->k_rmax, P->om, P->h, zo, rlo[j], rhi[j]);

    const int U = (int)ceil(rh / P->box) + 1;
    const double halfdiag = 0.5 * sqrt(3.0) * l;
    const double inv_s3 = 1.0 / ((double)S * S * S);
    /* one task per sorted octant cell a <= b <= c; the value is copied to
     * its permutations afterwards */
#pragma omp parallel
    {
        double* acc = (double*)malloc(sizeof(double) * A);
#pragma omp for schedule(dynamic, 16)
        for (int c = 0; c <= M; ++c) {
            for (int b = 0; b <= c; ++b) {
                for (int a = 0; a <= b; ++a) {
                    for (int j = 0; j < A; ++j) acc[j] = 0.0;
                    for (int u = -U; u <= U; ++u)
                        for (int v = -U; v <= U; ++v)
                            for (int w = -U; w <= U; ++w) {
                                double cx = l * (a + (double)u * N), cy = l * (b + (double)v * N),
                                       cz = l * (c + (double)w * N);
                                double dc = sqrt(cx * cx + cy * cy + cz * cz);
                                if (dc - halfdiag > rh) continue;
                                for (int sa = 0; sa < S; ++sa)
                                    for (int sb = 0; sb < S; ++sb)
                                        for (int sc = 0; sc < S; ++sc) {
                                            int64_t mx = 2LL * S * (a + (int64_t)u * N) + 2 * sa + 1 - S;
                                            int64_t my = 2LL * S * (b + (int64_t)v * N) + 2 * sb + 1 - S;
                                            int64_t mz = 2LL * S * (c + (int64_t)w * N) + 2 * sc + 1 - S;
                                            int64_t R = mx * mx + my * my + mz * mz;
                                            if (R > Rh || R < bnd[0] || R >= bnd[A]) continue;
                                            /* shell index: largest j with bnd[j] <= R */
                                            int lo = 0, hi = A; /* bnd[lo] <= R < bnd[hi] */
                                            while (hi - lo > 1) {
                                                int mid = (lo + hi) / 2;
                                                if (bnd[mid] <= R) lo = mid;
                                                else hi = mid;
                                            }
                                            acc[lo] += tab[(R - 3) / 8];
                                        }
                            }
                    int p[6][3] = {{a, b, c}, {a, c, b}, {b, a, c}, {b, c, a}, {c, a, b}, {c, b, a}};
                    for (int j = 0; j < A; ++j) {
                        double val = acc[j] * inv_s3;
                        double* G = out->G + (size_t)j * oct;
                        for (int q = 0; q < 6; ++q)
                            G[((size_t)p[q][0] * (M + 1) + p[q][1]) * (M + 1) + p[q][2]] = val;
                    }
                }
            }
        }
        free(acc);
    }
    /* full-grid sums: folded index x stands for 1 cell if x in {0, M}, else 2 */
    for (int j = 0; j < A; ++j) {
        const double* G = out->G + (size_t)j * oct;
        double sm = 0.0;
        for (int a = 0; a <= M; ++a)
            for (int b = 0; b <= M; ++b)
                for (int c = 0; c <= M; ++c) {
                    double mlt = (a == 0 || a == M ? 1.0 : 2.0) * (b == 0 || b == M ? 1.0 : 2.0) *
                                 (c == 0 || c == M ? 1.0 : 2.0);
                    sm += mlt * G[((size_t)a * (M + 1) + b) * (M + 1) + c];
                }
        out->sum[j] = sm;
        if (P->normalise && sm > 0.0) {
            double f = out->I[j] / (l * l * l * sm);
            double* Gm = out->G + (size_t)j * oct;
            for (size_t t = 0; t < oct; ++t) Gm[t] *= f;
        }
    }
    free(tab);
    free(bnd);
    free(rlo);
    free(rhi);
    return 0;
}

int lco_active_shells(const lco_problem* P, int s) { return lco_shells(P, s, NULL, NULL, NULL); }

/* The octant of G_j for step s (normalised if P->normalise), plus I_j and the
 * un-normalised full-grid sum. */
int lco_rgf_octant(const lco_problem* P, int s, int j, double* out, double* I, double* sum) {
    octant_set o;
    build_octants(P, s, &o);
    if (j < 0 || j >= o.A) {
        octant_free(&o);
        return 1;
    }
    size_t oct = (size_t)(o.M + 1) * (o.M + 1) * (o.M + 1);
    memcpy(out, o.G + (size_t)j * oct, sizeof(double) * oct);
    if (I) *I = o.I[j];
    if (sum) *sum = o.sum[j];
    octant_free(&o);
    return 0;
}

/* Un-normalised G_j at one displacement (dx, dy, dz), summed directly over
 * samples and images without any use of symmetry (a check on the octant). */
double lco_rgf_direct(const lco_problem* P, int s, int j, int dx, int dy, int dz) {
    const int N = P->n, S = P->subsamples;
    const double l = P->box / N, delta = l / (2.0 * S);
    double* rlo = (double*)malloc(sizeof(double) * (s + 1));
    double* rhi = (double*)malloc(sizeof(double) * (s + 1));
    double rh;
    int A = lco_shells(P, s, rlo, rhi, &rh);
    double res = 0.0;
    if (j >= 0 && j < A) {
        int64_t lo = ceil_i64((rlo[j] / delta) * (rlo[j] / delta));
        int64_t hi = ceil_i64((rhi[j] / delta) * (rhi[j] / delta));
        int64_t Rh = (int64_t)floor((rh / delta) * (rh / delta));
        const double zo = P->z_edges[s + 1];
        const int U = (int)ceil(rh / P->box) + 2;
        for (int u = -U; u <= U; ++u)
            for (int v = -U; v <= U; ++v)
                for (int w = -U; w <= U; ++w)
                    for (int sa = 0; sa < S; ++sa)
                        for (int sb = 0; sb < S; ++sb)
                            for (int sc = 0; sc < S; ++sc) {
                                int64_t mx = 2LL * S * (dx + (int64_t)u * N) + 2 * sa + 1 - S;
                                int64_t my = 2LL * S * (dy + (int64_t)v * N) + 2 * sb + 1 - S;
                                int64_t mz = 2LL * S * (dz + (int64_t)w * N) + 2 * sc + 1 - S;
                                int64_t R = mx * mx + my * my + mz * mz;
                                if (R < lo || R >= hi || R > Rh) continue;
                                res += lco_gk(P->kernel, P->k_length, P->k_rmax, P->om, P->h, zo,
                                              delta * sqrt((double)R));
                            }
        res /= (double)S * S * S;
    }
    free(rlo);
    free(rhi);
    return res;
}

/* ------------------------------------------------------------------ */
/* Source deposit (Eq. 11: l^3 absorbed into f_n; Eq. 17 source term)  */
/* ------------------------------------------------------------------ */
/* Nearest-grid-point cell of coordinate x: floor(x / l + 1/2) mod N, with
 * l = L / N, in IEEE double (the cell centre of index i sits at x = i l). */
static int64_t ngp_index(double x, double l, int N) {
    double t = floor(x / l + 0.5);
    double m = fmod(t, (double)N); /* exact */
    if (m < 0.0) m += (double)N;
    int64_t i = (int64_t)m;
    return (i >= 0 && i < N) ? i : 0;
}

static int check_sources(int64_t n_src, const double* pos, const double* lum) {
    for (int64_t s = 0; s < n_src; ++s) {
        if (!isfinite(lum[s]) || lum[s] < 0.0) return 2;
        for (int d = 0; d < 3; ++d)
            if (!isfinite(pos[3 * s + d])) return 2;
    }
    return 0;
}

/* FP64 luminosity per cell. */
int lco_deposit_ngp(int N, double box, int64_t n_src, const double* pos, const double* lum, double* grid) {
    int e = check_sources(n_src, pos, lum);
    if (e) return e;
    const double l = box / N;
    memset(grid, 0, sizeof(double) * (size_t)N * N * N);
    for (int64_t s = 0; s < n_src; ++s) {
        int64_t i = ngp_index(pos[3 * s + 0], l, N), j = ngp_index(pos[3 * s + 1], l, N),
                k = ngp_index(pos[3 * s + 2], l, N);
        grid[(i * N + j) * N + k] += lum[s];
    }
    return 0;
}

/* Integer fixed-point deposit: unit S = 2^(E - 62) with n_src * max(L) < 2^E,
 * q_s = rint(L_s / S); grid holds sum q per cell, *total the sum of all q.
 * Integer sums make the grid independent of source order. */
int lco_deposit_fixed(int N, double box, int64_t n_src, const double* pos, const double* lum, int64_t* grid,
                      double* scale, int64_t* total) {
    int e = check_sources(n_src, pos, lum);
    if (e) return e;
    const double l = box / N;
    memset(grid, 0, sizeof(int64_t) * (size_t)N * N * N);
    double lmax = 0.0;
    for (int64_t s = 0; s < n_src; ++s)
        if (lum[s] > lmax) lmax = lum[s];
    double S = 1.0;
    if (lmax > 0.0) {
        int E;
        frexp((double)n_src * lmax, &E);
        S = ldexp(1.0, E - 62);
    }
    int64_t tot = 0;
    for (int64_t s = 0; s < n_src; ++s) {
        int64_t q = (int64_t)rint(lum[s] / S);
        int64_t i = ngp_index(pos[3 * s + 0], l, N), j = ngp_index(pos[3 * s + 1], l, N),
                k = ngp_index(pos[3 * s + 2], l, N);
        grid[(i * N + j) * N + k] += q;
        tot += q;
    }
    *scale = S;
    *total = tot;
    return 0;
}

/* Cloud-in-cell assignment (an alternative to the nearest grid point for the
 * source term of Eq. 11 and Eq. 17): a source at coordinate x shares its
 * luminosity between the two cell centres around it along each axis, cells
 * i0 = floor(x / l) and i0 + 1 (mod N), with weights 1 - f and f,
 * f = x / l - floor(x / l); the 8 cells of a source get the products of the
 * per-axis weights (trilinear).  A source exactly at a cell centre (f = 0 on
 * every axis) puts everything in that cell, as the nearest grid point does. */
static void cic_axis(double x, double l, int N, int64_t* i0, int64_t* i1, double* f) {
    double t = x / l;
    double fl = floor(t);
    *f = t - fl;
    double m = fmod(fl, (double)N); /* exact */
    if (m < 0.0) m += (double)N;
    int64_t i = (int64_t)m;
    if (i < 0 || i >= N) i = 0;
    *i0 = i;
    *i1 = (i + 1) % N;
}

/* FP64 luminosity per cell, CIC weights. */
int lco_deposit_cic(int N, double box, int64_t n_src, const double* pos, const double* lum, double* grid) {
    int e = check_sources(n_src, pos, lum);
    if (e) return e;
    const double l = box / N;
    memset(grid, 0, sizeof(double) * (size_t)N * N * N);
    for (int64_t s = 0; s < n_src; ++s) {
        int64_t c[3][2];
        double w[3][2];
        for (int d = 0; d < 3; ++d) {
            double f;
            cic_axis(pos[3 * s + d], l, N, &c[d][0], &c[d][1], &f);
            w[d][0] = 1.0 - f;
            w[d][1] = f;
        }
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int k = 0; k < 2; ++k)
                    grid[(c[0][a] * N + c[1][b]) * N + c[2][k]] += lum[s] * w[0][a] * w[1][b] * w[2][k];
    }
    return 0;
}

/* Split an integer charge q >= 0 by weight f in [0, 1]: the part for the
 * upper cell, rint(q f) (at most q), and the rest for the lower one; the two
 * parts always sum to q. */
static void split_charge(int64_t q, double f, int64_t* lo, int64_t* hi) {
    int64_t h = (int64_t)rint((double)q * f);
    if (h > q) h = q;
    if (h < 0) h = 0;
    *hi = h;
    *lo = q - h;
}

/* Integer fixed-point CIC: the unit S and q_s = rint(L_s / S) as
 * lco_deposit_fixed; each q_s is split along x, then each part along y, then
 * each of those along z (split_charge), so the 8 integer charges of a source
 * sum to q_s exactly and the grid total equals the sum of all q_s. */
int lco_deposit_cic_fixed(int N, double box, int64_t n_src, const double* pos, const double* lum, int64_t* grid,
                          double* scale, int64_t* total) {
    int e = check_sources(n_src, pos, lum);
    if (e) return e;
    const double l = box / N;
    memset(grid, 0, sizeof(int64_t) * (size_t)N * N * N);
    double lmax = 0.0;
    for (int64_t s = 0; s < n_src; ++s)
        if (lum[s] > lmax) lmax = lum[s];
    double S = 1.0;
    if (lmax > 0.0) {
        int E;
        frexp((double)n_src * lmax, &E);
        S = ldexp(1.0, E - 62);
    }
    int64_t tot = 0;
    for (int64_t s = 0; s < n_src; ++s) {
        int64_t q = (int64_t)rint(lum[s] / S);
        int64_t c[3][2];
        double f[3];
        for (int d = 0; d < 3; ++d) cic_axis(pos[3 * s + d], l, N, &c[d][0], &c[d][1], &f[d]);
        int64_t qx[2], qxy[2][2], qxyz[2][2][2];
        split_charge(q, f[0], &qx[0], &qx[1]);
        for (int a = 0; a < 2; ++a) {
            split_charge(qx[a], f[1], &qxy[a][0], &qxy[a][1]);
            for (int b = 0; b < 2; ++b) split_charge(qxy[a][b], f[2], &qxyz[a][b][0], &qxyz[a][b][1]);
        }
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int k = 0; k < 2; ++k) grid[(c[0][a] * N + c[1][b]) * N + c[2][k]] += qxyz[a][b][k];
        tot += q;
    }
    *scale = S;
    *total = tot;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Retarded field by direct periodic convolution (Eq. 11), summed over  */
/* slices (Eq. 9, step 6 of Section 2.2).                              */
/* ------------------------------------------------------------------ */
/* The sum of Eq. 11 over slices at the requested cells, from the occupied
 * cells of each slice: slice j (lookback j, j < n_slices) has counts[j]
 * entries, flat C-order cell indices flat[] and FP64 values val[], the slices'
 * entries concatenated in order of j.  cells: flat indices to evaluate, or
 * NULL for all N^3.  Slices at or beyond the step's active count add
 * nothing. */
static int field_sum(const lco_problem* P, int s, int n_slices, const int64_t* counts, const int64_t* flat,
                     const double* val, int64_t n_cells, const int64_t* cells, double* out) {
    const int N = P->n, M = N / 2;
    const size_t NN = (size_t)N * N * N;
    octant_set o;
    if (build_octants(P, s, &o)) return 1;
    const size_t oct = (size_t)(M + 1) * (M + 1) * (M + 1);
    const int A = o.A < n_slices ? o.A : n_slices;
    int64_t* occ_start = (int64_t*)calloc(A + 1, sizeof(int64_t));
    for (int j = 0; j < A; ++j) occ_start[j + 1] = occ_start[j] + counts[j];
    const int64_t total_occ = occ_start[A];
    int* oi = (int*)malloc(sizeof(int) * (total_occ + 1));
    int* oj = (int*)malloc(sizeof(int) * (total_occ + 1));
    int* ok = (int*)malloc(sizeof(int) * (total_occ + 1));
    for (int64_t p = 0; p < total_occ; ++p) {
        const int64_t t = flat[p];
        oi[p] = (int)(t / ((int64_t)N * N));
        oj[p] = (int)((t / N) % N);
        ok[p] = (int)(t % N);
    }
    const int64_t nc = cells ? n_cells : (int64_t)NN;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t c = 0; c < nc; ++c) {
        int64_t t = cells ? cells[c] : c;
        int x = (int)(t / ((int64_t)N * N)), y = (int)((t / N) % N), z = (int)(t % N);
        double acc = 0.0;
        for (int j = 0; j < A; ++j) {
            const double* G = o.G + (size_t)j * oct;
            for (int64_t p = occ_start[j]; p < occ_start[j + 1]; ++p) {
                int dx = ((x - oi[p]) % N + N) % N, dy = ((y - oj[p]) % N + N) % N, dz = ((z - ok[p]) % N + N) % N;
                if (dx > M) dx = N - dx;
                if (dy > M) dy = N - dy;
                if (dz > M) dz = N - dz;
                acc += G[((size_t)dx * (M + 1) + dy) * (M + 1) + dz] * val[p];
            }
        }
        out[c] = P->out_unit * acc;
    }
    free(oi);
    free(oj);
    free(ok);
    free(occ_start);
    octant_free(&o);
    return 0;
}

/* src[j] is the FP64 source grid of slice s - j (NULL: no sources), for
 * j < n_src_grids.  cells: flat C-order indices, or NULL for all N^3.  The
 * occupied cells of each grid, in increasing flat index, go to field_sum. */
int lco_field(const lco_problem* P, int s, int n_src_grids, const double* const* src, int64_t n_cells,
              const int64_t* cells, double* out) {
    const int N = P->n;
    const size_t NN = (size_t)N * N * N;
    const int ns = n_src_grids > 0 ? n_src_grids : 0;
    int64_t* counts = (int64_t*)calloc(ns + 1, sizeof(int64_t));
    int64_t total = 0;
    for (int j = 0; j < ns; ++j) {
        if (src[j])
            for (size_t t = 0; t < NN; ++t)
                if (src[j][t] != 0.0) ++counts[j];
        total += counts[j];
    }
    int64_t* flat = (int64_t*)malloc(sizeof(int64_t) * (total + 1));
    double* val = (double*)malloc(sizeof(double) * (total + 1));
    int64_t p = 0;
    for (int j = 0; j < ns; ++j)
        if (src[j])
            for (size_t t = 0; t < NN; ++t)
                if (src[j][t] != 0.0) {
                    flat[p] = (int64_t)t;
                    val[p] = src[j][t];
                    ++p;
                }
    int rc = field_sum(P, s, ns, counts, flat, val, n_cells, cells, out);
    free(counts);
    free(flat);
    free(val);
    return rc;
}

/* The same field from the slices' occupied-cell lists (see field_sum), for
 * grids too large to hold every slice's dense grid at once. */
int lco_field_sparse(const lco_problem* P, int s, int n_slices, const int64_t* counts, const int64_t* flat,
                     const double* val, int64_t n_cells, const int64_t* cells, double* out) {
    return field_sum(P, s, n_slices, counts, flat, val, n_cells, cells, out);
}

/* Shell integrals I_j (Green's-function k = 0 values times l^3) of step s. */
/* Near field of the innermost slice from the sources' own positions (the
 * particle-mesh hybrid the Discussion suggests for sources resolved below the
 * mesh).  For every source of the observing step's own slice (j = 0) and
 * every target cell within R cells (per axis) of the source's NGP cell, add
 *   U * lum * f0 / s^3 * sum_{s^3 sub-samples y of the target cell}
 *        sum_{periodic images u} [r < r_hi(0), r <= r_h] g(r),   r = |y - x_src + u L|,
 * to out (N^3, C order, accumulated): the same sub-sampled shell average as
 * G_0 (Eq. 10), with f0 its normalisation factor, but centred on the source
 * position instead of its cell.  centred != 0 puts every source at its cell
 * centre, which gives back U * lum * G_0(target - cell) exactly: the near
 * cube of the NGP field. */
int lco_near_cube(const lco_problem* P, int s, int64_t n_src, const double* pos, const double* lum, int R,
                  double f0, int centred, double* out) {
    const int N = P->n, S = P->subsamples;
    const double l = P->box / N, L = P->box;
    const double zo = P->z_edges[s + 1];
    double rlo[1], rhi[1], rh;
    if (s < 0 || s >= P->n_steps) return 1;
    double* lo_all = (double*)malloc(sizeof(double) * (s + 1));
    double* hi_all = (double*)malloc(sizeof(double) * (s + 1));
    int A = lco_shells(P, s, lo_all, hi_all, &rh);
    if (A <= 0) {
        free(lo_all);
        free(hi_all);
        return 0;
    }
    rlo[0] = lo_all[0];
    rhi[0] = hi_all[0];
    free(lo_all);
    free(hi_all);
    const double top = rhi[0];
    const int U = (int)ceil((top + 2.0 * (R + 1) * l) / L) + 1;
    const double wgt = P->out_unit * f0 / ((double)S * S * S);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < n_src; ++q) {
        const double x[3] = {pos[3 * q], pos[3 * q + 1], pos[3 * q + 2]};
        int64_t c[3];
        double off[3];
        for (int d = 0; d < 3; ++d) {
            c[d] = ngp_index(x[d], l, N);
            /* the source relative to its cell centre, in [-l/2, l/2) */
            double t = x[d] / l + 0.5;
            off[d] = centred ? 0.0 : (t - floor(t) - 0.5) * l;
        }
        const double halfdiag = 0.5 * sqrt(3.0) * l;
        for (int dx = -R; dx <= R; ++dx)
            for (int dy = -R; dy <= R; ++dy)
                for (int dz = -R; dz <= R; ++dz) {
                    double acc = 0.0;
                    for (int u = -U; u <= U; ++u)
                        for (int v = -U; v <= U; ++v)
                            for (int w = -U; w <= U; ++w) {
                                /* target cell centre minus source, this image */
                                double cx = l * dx - off[0] + u * L, cy = l * dy - off[1] + v * L,
                                       cz = l * dz - off[2] + w * L;
                                /* every sample is within halfdiag of the centre */
                                if (sqrt(cx * cx + cy * cy + cz * cz) - halfdiag >= top) continue;
                                for (int a = 0; a < S; ++a)
                                    for (int b = 0; b < S; ++b)
                                        for (int e = 0; e < S; ++e) {
                                            double px = cx + l * ((a + 0.5) / S - 0.5);
                                            double py = cy + l * ((b + 0.5) / S - 0.5);
                                            double pz = cz + l * ((e + 0.5) / S - 0.5);
                                            double r = sqrt(px * px + py * py + pz * pz);
                                            if (!(r >= rlo[0] && r < top && r <= rh)) continue;
                                            acc += lco_gk(P->kernel, P->k_length, P->k_rmax, P->om, P->h, zo, r);
                                        }
                            }
                    int64_t tx = ((c[0] + dx) % N + N) % N, ty = ((c[1] + dy) % N + N) % N,
                            tz = ((c[2] + dz) % N + N) % N;
                    double val = wgt * lum[q] * acc;
#pragma omp atomic
                    out[(tx * N + ty) * N + tz] += val;
                }
    }
    return 0;
}

int lco_shell_table(const lco_problem* P, int s, double* r_lo, double* r_hi, double* I) {
    int A = lco_shells(P, s, r_lo, r_hi, NULL);
    double zo = P->z_edges[s + 1];
    for (int j = 0; j < A; ++j)
        I[j] = lco_shell_integralk(P->kernel, P->k_length, P->k_rmax, P->om, P->h, zo, r_lo[j], r_hi[j]);
    return A;
}

/* ------------------------------------------------------------------ */
/* Brute-force 3D DFT (Eq. 12 convention): X(p) = sum x(i) e^{sign 2 pi i p.i / N}, */
/* unnormalised; the inverse of Eq. 12 is sign = +1 followed by 1/N^3.             */
/* ------------------------------------------------------------------ */
int lco_dft3(int N, const double* re, const double* im, int sign, double* ore, double* oim) {
    double* c = (double*)malloc(sizeof(double) * N);
    double* sn = (double*)malloc(sizeof(double) * N);
    for (int m = 0; m < N; ++m) {
        c[m] = cos(2.0 * OR_PI * m / N);
        sn[m] = sin(2.0 * OR_PI * m / N);
    }
    const size_t NN = (size_t)N * N * N;
#pragma omp parallel for schedule(static)
    for (size_t P = 0; P < NN; ++P) {
        int p = (int)(P / ((size_t)N * N)), q = (int)((P / N) % N), r = (int)(P % N);
        double sr = 0.0, si = 0.0;
        for (size_t T = 0; T < NN; ++T) {
            int i = (int)(T / ((size_t)N * N)), j = (int)((T / N) % N), k = (int)(T % N);
            int m = (int)(((int64_t)i * p + (int64_t)j * q + (int64_t)k * r) % N);
            double cr = c[m], ci = sign * sn[m];
            double xr = re[T], xi = im ? im[T] : 0.0;
            sr += xr * cr - xi * ci;
            si += xr * ci + xi * cr;
        }
        ore[P] = sr;
        oim[P] = si;
    }
    free(c);
    free(sn);
    return 0;
}

int lco_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
