// lc_host.cpp -- host FP64 planning for the retarded-field path: flat-LCDM
// cosmology (Eqs. 5-6), the LW kernel constants (Eqs. 15-16), the time
// slicing (step 1 of Section 2.2, Eq. 9) and the integer shell geometry used
// by the Green's function builder (Eq. 10).  Everything here runs once per
// plan or per observing step, never in the per-step hot path.
#include <math.h>

#include <algorithm>
#include <vector>

#include "lc_internal.h"

namespace lc {
namespace {

constexpr double kC = 299792.458;          // km/s
constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kMpcKm = 3.0856775814913673e19;
constexpr double kMyrSec = 3.15576e13;

// 12-point Gauss-Legendre nodes/weights on [-1, 1], found by Newton's method
// on the Legendre recurrence.
struct GaussLegendre12 {
    double x[12], w[12];
    GaussLegendre12() {
        const int n = 12;
        for (int i = 0; i < n; ++i) {
            double r = cos(kPi * (i + 0.75) / (n + 0.5)), d = 1.0;
            for (int it = 0; it < 60; ++it) {
                double pm = 1.0, p = r; // P_{k-1}, P_k
                for (int k = 2; k <= n; ++k) {
                    double pn = ((2 * k - 1) * r * p - (k - 1) * pm) / k;
                    pm = p;
                    p = pn;
                }
                d = n * (pm - r * p) / (1.0 - r * r);
                double step = p / d;
                r -= step;
                if (fabs(step) < 5e-17) break;
            }
            x[i] = r;
            w[i] = 2.0 / ((1.0 - r * r) * d * d);
        }
    }
};
const GaussLegendre12& gl() {
    static const GaussLegendre12 g;
    return g;
}

inline double inv_h(const Cosmo& c, double z) { return kC / hubble(c, z); }

// int_a^b c/H dz on one panel
double chi_panel(const Cosmo& c, double a, double b) {
    const GaussLegendre12& q = gl();
    const double m = 0.5 * (a + b), hw = 0.5 * (b - a);
    double s = 0.0;
    for (int i = 0; i < 12; ++i) s += q.w[i] * inv_h(c, m + hw * q.x[i]);
    return hw * s;
}

} // namespace

double hubble(const Cosmo& c, double z) {
    const double a = 1.0 + z;
    return 100.0 * c.h * sqrt(c.om * a * a * a + (1.0 - c.om));
}

double chi(const Cosmo& c, double z1, double z2) {
    if (z1 == z2) return 0.0;
    if (z2 < z1) return -chi(c, z2, z1);
    const int np = std::max(1, (int)ceil((z2 - z1) / 0.1));
    const double w = (z2 - z1) / np;
    double s = 0.0;
    for (int p = 0; p < np; ++p) s += chi_panel(c, z1 + p * w, z1 + (p + 1) * w);
    return s;
}

double time_myr(const Cosmo& c, double z) {
    const double tH = kMpcKm / (100.0 * c.h) / kMyrSec;
    const double ol = 1.0 - c.om, y = pow(1.0 + z, -1.5);
    if (ol <= 0.0) return (2.0 / 3.0) * tH * y;
    return (2.0 / 3.0) * tH / sqrt(ol) * asinh(sqrt(ol / c.om) * y);
}

double z_of_time(const Cosmo& c, double t) {
    const double tH = kMpcKm / (100.0 * c.h) / kMyrSec;
    const double ol = 1.0 - c.om;
    const double y = ol <= 0.0 ? 1.5 * t / tH : sinh(1.5 * sqrt(ol) * t / tH) * sqrt(c.om / ol);
    return pow(y, -2.0 / 3.0) - 1.0;
}

double zs_of_r(const Cosmo& c, double zo, double r) {
    if (r <= 0.0) return zo;
    // matter-dominated first guess, then Newton on chi(zo, z) = r with
    // d chi / dz = c / H; the bracket keeps it safe.
    const double H0 = 100.0 * c.h;
    double x = 1.0 / sqrt(1.0 + zo) - r * H0 * sqrt(c.om) / (2.0 * kC);
    double z = x > 0.05 ? 1.0 / (x * x) - 1.0 : zo + 10.0;
    double lo = zo, hi = 1e9;
    for (int it = 0; it < 100; ++it) {
        const double f = chi(c, zo, z) - r;
        if (f > 0) hi = std::min(hi, z);
        else lo = std::max(lo, z);
        double zn = z - f / inv_h(c, z);
        if (!(zn > lo && zn < hi)) zn = hi < 1e9 ? 0.5 * (lo + hi) : 2.0 * z - zo + 1.0;
        if (fabs(zn - z) <= 4e-16 * (1.0 + z)) return zn;
        z = zn;
    }
    return z;
}

double alpha_lw(const Cosmo& c, double zs) {
    return (0.7 / c.h) / sqrt(c.om / 0.27) / sqrt((1.0 + zs) / 21.0);
}

double fmod_lw(double r, double alpha) {
    if (r > 97.39 * alpha) return 0.0;
    return 1.7 * exp(-pow(r / (116.29 * alpha), 0.68)) - 0.7;
}

double rough_horizon(double zs) { return 100.0 * sqrt(21.0 / (1.0 + zs)); }

double kernel_f(const Cosmo& c, const Kernel& k, double zs, double r) {
    if (k.kind == LC_KERNEL_EXP) return r < k.rmax ? exp(-r / k.length) : 0.0;
    if (k.kind == kKernelLwRough) {
        // Eq. 15's modulation without its cut, clamped at 0, inside the rough horizon
        if (r > rough_horizon(zs)) return 0.0;
        const double f = 1.7 * exp(-pow(r / (116.29 * alpha_lw(c, zs)), 0.68)) - 0.7;
        return f > 0.0 ? f : 0.0;
    }
    return fmod_lw(r, alpha_lw(c, zs));
}

namespace {
// the radius r (seen from z_obs) where r = h(z_s(r)) for a function h that
// falls as z_s grows: bisection from [0, h(z_obs)]
template <class H> double light_cone_root(const Cosmo& c, double zo, H h) {
    double a = 0.0, b = h(zo);
    for (int it = 0; it < 120 && b - a > 1e-14 * b; ++it) {
        const double m = 0.5 * (a + b);
        if (m - h(zs_of_r(c, zo, m)) > 0.0) b = m;
        else a = m;
    }
    return 0.5 * (a + b);
}
// kKernelLwRough: where the unclamped modulation of Eq. 15 reaches 0,
// r = 116.29 ln(1.7 / 0.7)^(1 / 0.68) alpha(z_s(r))
double fmod_zero_radius(const Cosmo& c, double zo) {
    const double x0 = 116.29 * pow(log(1.7 / 0.7), 1.0 / 0.68);
    return light_cone_root(c, zo, [&](double zs) { return x0 * alpha_lw(c, zs); });
}
} // namespace

double horizon(const Cosmo& c, const Kernel& k, double zo) {
    if (k.kind == LC_KERNEL_EXP) return k.rmax;
    if (k.kind == kKernelLwRough) return light_cone_root(c, zo, [](double zs) { return rough_horizon(zs); });
    return light_cone_root(c, zo, [&](double zs) { return 97.39 * alpha_lw(c, zs); });
}

namespace {
double shell_integrand(const Cosmo& c, const Kernel& k, double zo, double r) {
    const double zs = zs_of_r(c, zo, r);
    const double o = 1.0 + zo;
    return o * o * o * kernel_f(c, k, zs, r) / (4.0 * kPi * (1.0 + zs));
}
double gl_integral(const Cosmo& c, const Kernel& k, double zo, double a, double b) {
    const GaussLegendre12& q = gl();
    const double m = 0.5 * (a + b), hw = 0.5 * (b - a);
    double s = 0.0;
    for (int i = 0; i < 12; ++i) s += q.w[i] * shell_integrand(c, k, zo, m + hw * q.x[i]);
    return hw * s;
}
} // namespace

double shell_integral(const Cosmo& c, const Kernel& kern, double zo, double r_lo, double r_hi, double r_h) {
    double b = std::min(r_hi, r_h);
    // the clamped kernel is 0 beyond its zero: stop there, so that no
    // quadrature panel straddles the kink
    if (kern.kind == kKernelLwRough) b = std::min(b, fmod_zero_radius(c, zo));
    if (!(r_lo < b)) return 0.0;
    double s = 0.0;
    if (r_lo <= 0.0) {
        // f_mod carries r^0.68 at the origin: geometric panels [b/2^(k+1), b/2^k]
        for (int k = 0; k < 56; ++k) s += gl_integral(c, kern, zo, ldexp(b, -(k + 1)), ldexp(b, -k));
        return s;
    }
    double x = r_lo;
    while (x < b) {
        double w = std::min(0.5 * x, 2.0);
        if (x + w > b) w = b - x;
        s += gl_integral(c, kern, zo, x, x + w);
        x += w;
    }
    return s;
}

int step_edges(const Cosmo& c, const Kernel& k, const lc_steps& st, std::vector<double>& z) {
    const int n = st.n_steps;
    if (n < 1) return 1;
    z.assign(n + 1, 0.0);
    if (st.spacing == LC_STEPS_EXPLICIT) {
        if (!st.z_edges) return 1;
        for (int k = 0; k <= n; ++k) z[k] = st.z_edges[k];
    } else if (st.spacing == LC_STEPS_EQUAL_TIME) {
        const double t0 = time_myr(c, st.z_start), t1 = time_myr(c, st.z_end);
        for (int k = 0; k <= n; ++k) z[k] = z_of_time(c, t0 + (t1 - t0) * k / n);
        z[0] = st.z_start;
        z[n] = st.z_end;
    } else if (st.spacing == LC_STEPS_EQUAL_TAU) {
        if (st.n_shell < 1) return 1;
        const double dtau = horizon(c, k, st.z_end) / st.n_shell;
        for (int k = 0; k < n; ++k) z[k] = zs_of_r(c, st.z_end, (n - k) * dtau);
        z[n] = st.z_end;
    } else {
        return 1;
    }
    for (int k = 0; k < n; ++k)
        if (!(z[k] > z[k + 1]) || !std::isfinite(z[k]) || z[k + 1] < 0.0) return 1;
    return 0;
}

void g_table(const Cosmo& c, const Kernel& k, double zo, double delta, long long ntab, double* out) {
    // Walk outwards in r; z_s(r) follows from the previous point by Newton on
    // the increment chi(z_prev, z) (one Gauss-Legendre panel), re-anchored on
    // the full distance every 512 entries so that rounding cannot drift.
    const double o3 = (1.0 + zo) * (1.0 + zo) * (1.0 + zo);
    const double k16pi2 = 16.0 * kPi * kPi;
    double r_prev = 0.0, z_prev = zo;
    for (long long t = 0; t < ntab; ++t) {
        const double r = delta * sqrt((double)(8 * t + 3));
        double z = z_prev + (r - r_prev) / inv_h(c, z_prev);
        for (int it = 0; it < 8; ++it) {
            const double f = r_prev + chi_panel(c, z_prev, z) - r;
            const double dz = f / inv_h(c, z);
            z -= dz;
            if (fabs(dz) <= 2e-16 * (1.0 + z)) break;
        }
        if ((t & 511) == 511) {
            z = zs_of_r(c, zo, r);
        }
        r_prev = r;
        z_prev = z;
        const double fm = kernel_f(c, k, z, r);
        out[t] = fm > 0.0 ? o3 * fm / (k16pi2 * (1.0 + z) * r * r) : 0.0;
    }
}

StepGeom step_geometry(const Cosmo& c, const Kernel& k, const std::vector<double>& z, int s, double l, int S,
                       bool integrals, int cap) {
    StepGeom g;
    const double zo = z[s + 1];
    g.rh = horizon(c, k, zo);
    for (int j = 0; j <= s; ++j) {
        if (cap > 0 && j >= cap) break; // the newest `cap` slices only
        const int n = s - j;
        const double lo = chi(c, zo, z[n + 1]);
        const double hi = chi(c, zo, z[n]);
        // a slice whose inner radius reaches the horizon (to 1e-9) carries no weight
        if (!(lo < g.rh * (1.0 - 1e-9))) break;
        g.lo.push_back(lo);
        g.hi.push_back(hi);
    }
    g.A = (int)g.lo.size();
    const double delta = l / (2.0 * S);
    // sample with integer squared radius R (units delta^2) is in shell j iff
    // bnd[j] <= R < bnd[j+1], i.e. r_lo <= r < r_hi exactly
    g.bnd.resize(g.A + 1);
    if (g.A > 0) {
        g.bnd[0] = (long long)ceil((g.lo[0] / delta) * (g.lo[0] / delta));
        for (int j = 0; j < g.A; ++j) g.bnd[j + 1] = (long long)ceil((g.hi[j] / delta) * (g.hi[j] / delta));
    }
    g.Rh = (long long)floor((g.rh / delta) * (g.rh / delta));
    g.ntab = g.Rh >= 3 ? (g.Rh - 3) / 8 + 1 : 0;
    if (integrals) {
        g.I.resize(g.A);
        for (int j = 0; j < g.A; ++j) g.I[j] = shell_integral(c, k, zo, g.lo[j], g.hi[j], g.rh);
    }
    return g;
}

} // namespace lc
