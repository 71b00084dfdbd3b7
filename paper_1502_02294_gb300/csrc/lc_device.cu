// lc_device.cu -- source deposit and Green's function builder kernels.
//
// Deposit (Eq. 11 with l^3 absorbed into f_n; Eq. 17 source term): nearest
// grid point or cloud in cell, integer fixed point.  The unit S = 2^(E - 62)
// with n_src * max(L) < 2^E bounds every cell and the total below
// 2^62 + n_src/2; q_s = rint(L_s / S) (or, for cloud in cell, its 8 integer
// shares, which sum to q_s exactly) is added with 64-bit integer atomics, so
// the grid and the total are bit-exact and independent of source order.
//
// Green's function builder (Eq. 10, step 2 of Section 2.2): for every cell
// displacement on the symmetric wedge 0 <= a <= b <= c <= N/2, sum the LW
// kernel g(r) (Eq. 17) over s^3 sub-cell samples and all periodic images of
// the unit source; a sample with integer squared radius R (units of
// (l / 2s)^2) belongs to shell j iff bnd[j] <= R < bnd[j+1] and counts iff
// R <= Rh (the horizon).  g is read from a table indexed by (R - 3) / 8.
#include <cuda_runtime.h>
#include <math.h>

#include "lc_fft.cuh"
#include "lc_internal.h"

namespace lc {
namespace {

constexpr int kPrepThreads = 1024;

__device__ __forceinline__ bool finite_d(double x) { return isfinite(x); }

__global__ void __launch_bounds__(kPrepThreads)
    k_src_prep(const double* __restrict__ pos, const double* __restrict__ lum, long long n,
               unsigned long long* maxbits, int* err, SlotMeta m) {
    __shared__ unsigned long long s_max[kPrepThreads / 32];
    __shared__ int s_bad;
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    // the luminosities only (positions are checked where they are used, in
    // k_deposit), four loads in flight per thread
    unsigned long long mx = 0;
    int bad = 0;
    for (long long i0 = threadIdx.x; i0 < n; i0 += 4 * kPrepThreads) {
        unsigned long long B[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long long i = i0 + (long long)u * kPrepThreads;
            B[u] = i < n ? (unsigned long long)__double_as_longlong(lum[i]) : 0ULL;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            // on the bit patterns (integer work; FP64 issue is narrow): finite
            // and >= 0 is a clear sign bit below the infinity pattern, or -0;
            // non-negative doubles order like their bit patterns
            if (B[u] < 0x7ff0000000000000ULL) mx = max(mx, B[u]);
            else if (B[u] != 0x8000000000000000ULL) bad = 1;
        }
    }
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = mx;
    if (bad) atomicOr(&s_bad, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long r = 0;
        for (int w = 0; w < kPrepThreads / 32; ++w) r = max(r, s_max[w]);
        *maxbits = r;
        if (s_bad) atomicOr(err, 1);
        m.slot_step[m.slot] = m.step;
        m.slot_total[m.slot] = 0;
        m.slot_S[m.slot] = 1.0; // replaced by the deposit's unit when there are sources
        if (m.stamp) *m.stamp += 1u;
    }
}

// t mod N for an integer-valued double t, in [0, N).  Below 2^53 in
// magnitude t converts to an integer exactly and the remainder is taken in
// integers; beyond, by fmod (exact as well).  FP64 issues at a small fraction
// of the FP32 rate on this GPU, and fmod is a loop of FP64 operations, so the
// integer path matters for the deposit's throughput.
__device__ __forceinline__ long long wrap_cell(double t, int N) {
    long long i;
    if (fabs(t) < 9007199254740992.0) {
        i = (long long)t % N;
        if (i < 0) i += N;
    } else {
        double m = fmod(t, (double)N);
        if (m < 0.0) m += (double)N;
        i = (long long)m;
    }
    return (i >= 0 && i < N) ? i : 0;
}

__device__ __forceinline__ long long ngp_cell(double x, double l, int N) {
    // floor(x / l + 1/2) mod N in IEEE double, no contraction
    return wrap_cell(floor(__dadd_rn(__ddiv_rn(x, l), 0.5)), N);
}

// Cloud in cell along one axis: the cells i0 = floor(x / l) mod N and
// i0 + 1 (mod N) around x, and the weight f = x / l - floor(x / l) of the
// upper one, in IEEE double (fmod exact, no contraction).
__device__ __forceinline__ void cic_axis(double x, double l, int N, long long& i0, long long& i1, double& f) {
    const double t = __ddiv_rn(x, l);
    const double fl = floor(t);
    f = __dsub_rn(t, fl);
    const long long i = wrap_cell(fl, N);
    i0 = i;
    i1 = i + 1 == N ? 0 : i + 1;
}

// Split an integer share q >= 0 by weight f: the upper cell's part
// min(q, rint(q f)), the lower cell's the rest (the two always sum to q).
__device__ __forceinline__ void split_share(long long q, double f, long long& lo, long long& hi) {
    long long h = __double2ll_rn(__dmul_rn(__ll2double_rn(q), f));
    h = h > q ? q : (h < 0 ? 0 : h);
    hi = h;
    lo = q - h;
}

template <int CIC>
__global__ void __launch_bounds__(256)
    k_deposit(const double* __restrict__ pos, const double* __restrict__ lum, long long n, int N, double l,
              const unsigned long long* __restrict__ maxbits, long long* __restrict__ grid, SlotMeta m, int* err,
              long long* __restrict__ cell_out, long long* __restrict__ q_out, double* __restrict__ off_out) {
    __shared__ long long s_sum[8];
    const double lmax = __longlong_as_double((long long)*maxbits);
    double S = 1.0, invS = 1.0;
    if (lmax > 0.0) {
        int E;
        frexp(__dmul_rn((double)n, lmax), &E);
        S = ldexp(1.0, E - 62);
        // L / S for a power of two S is the exact L 2^(62-E) rounded once, so
        // the product with 1/S is the same double whenever 1/S is a normal
        // number (E - 62 within the normal exponent range both ways)
        invS = (E - 62 > -1022 && E - 62 < 1022) ? ldexp(1.0, 62 - E) : 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) m.slot_S[m.slot] = S;
    // this push's value of the counter, stored for every row deposited into
    const unsigned stamp = m.rowstamp ? *m.stamp : 0u;
    long long q = 0;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const double L = lum[i];
        const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
        const bool ok = finite_d(L) && L >= 0.0 && finite_d(x) && finite_d(y) && finite_d(z);
        if (!ok) atomicOr(err, 1); // an invalid source is left out and reported
        if constexpr (CIC) {
            long long cx[2] = {0, 0}, cy[2] = {0, 0}, cz[2] = {0, 0};
            long long sh[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            if (ok) {
                q = llrint(invS != 0.0 ? __dmul_rn(L, invS) : __ddiv_rn(L, S));
                double fx, fy, fz;
                cic_axis(x, l, N, cx[0], cx[1], fx);
                cic_axis(y, l, N, cy[0], cy[1], fy);
                cic_axis(z, l, N, cz[0], cz[1], fz);
                // split along x, then each part along y, then each of those along z
                long long qx[2], qxy[4];
                split_share(q, fx, qx[0], qx[1]);
                for (int a = 0; a < 2; ++a) split_share(qx[a], fy, qxy[2 * a], qxy[2 * a + 1]);
                for (int ab = 0; ab < 4; ++ab) split_share(qxy[ab], fz, sh[2 * ab], sh[2 * ab + 1]);
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const long long c = (cx[k >> 2] * N + cy[(k >> 1) & 1]) * N + cz[k & 1];
                if (sh[k]) {
                    atomicAdd(reinterpret_cast<unsigned long long*>(grid + c), (unsigned long long)sh[k]);
                    if (m.rowstamp) m.rowstamp[c / N] = stamp;
                }
                if (cell_out) {
                    cell_out[8 * i + k] = c;
                    q_out[8 * i + k] = sh[k];
                }
            }
        } else {
            long long c = 0;
            if (ok) {
                q = llrint(invS != 0.0 ? __dmul_rn(L, invS) : __ddiv_rn(L, S));
                c = (ngp_cell(x, l, N) * N + ngp_cell(y, l, N)) * N + ngp_cell(z, l, N);
                if (q) {
                    atomicAdd(reinterpret_cast<unsigned long long*>(grid + c), (unsigned long long)q);
                    if (m.rowstamp) m.rowstamp[c / N] = stamp;
                }
            }
            if (cell_out) {
                cell_out[i] = c;
                q_out[i] = q;
            }
        }
        if (off_out) {
            // the source relative to its cell centre, in [-l/2, l/2) per axis
            const double p3[3] = {x, y, z};
            for (int d = 0; d < 3; ++d) {
                const double t = p3[d] / l + 0.5;
                off_out[3 * i + d] = finite_d(t) ? (t - floor(t) - 0.5) * l : 0.0;
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = q;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_sum[w];
        if (t) atomicAdd(reinterpret_cast<unsigned long long*>(m.slot_total + m.slot), (unsigned long long)t);
    }
}

// wedge index -> sorted triple a <= b <= c
__device__ __forceinline__ void wedge_decode(long long w, int& a, int& b, int& c) {
    int cc = (int)cbrt(6.0 * (double)w);
    while ((long long)(cc + 1) * (cc + 2) * (cc + 3) / 6 <= w) ++cc;
    while (cc > 0 && (long long)cc * (cc + 1) * (cc + 2) / 6 > w) --cc;
    long long rem = w - (long long)cc * (cc + 1) * (cc + 2) / 6;
    int bb = (int)((sqrt(8.0 * (double)rem + 1.0) - 1.0) * 0.5);
    while ((long long)(bb + 1) * (bb + 2) / 2 <= rem) ++bb;
    while (bb > 0 && (long long)bb * (bb + 1) / 2 > rem) --bb;
    a = (int)(rem - (long long)bb * (bb + 1) / 2);
    b = bb;
    c = cc;
}

constexpr int kMaxBnd = 1025;

__global__ void __launch_bounds__(128) k_rgf_accum(RgfAccumArgs a) {
    __shared__ long long s_bnd[kMaxBnd];
    for (int i = threadIdx.x; i <= a.A; i += blockDim.x) s_bnd[i] = a.bnd[i];
    __syncthreads();
    const long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= a.W) return;
    int ia, ib, ic;
    wedge_decode(w, ia, ib, ic);
    const int N = a.N, S = a.S, U = a.U;
    const double hd = 0.8660254037844386 * a.l;
    const long long top = s_bnd[a.A];
    for (int u = -U; u <= U; ++u)
        for (int v = -U; v <= U; ++v)
            for (int ww = -U; ww <= U; ++ww) {
                const double cx = a.l * (ia + (double)u * N), cy = a.l * (ib + (double)v * N),
                             cz = a.l * (ic + (double)ww * N);
                if (sqrt(cx * cx + cy * cy + cz * cz) - hd > a.rh) continue;
                const long long bx = 2LL * S * (ia + (long long)u * N) + 1 - S;
                const long long by = 2LL * S * (ib + (long long)v * N) + 1 - S;
                const long long bz = 2LL * S * (ic + (long long)ww * N) + 1 - S;
                for (int sa = 0; sa < S; ++sa) {
                    const long long mx = bx + 2 * sa, mx2 = mx * mx;
                    for (int sb = 0; sb < S; ++sb) {
                        const long long my = by + 2 * sb, mxy = mx2 + my * my;
                        for (int sc = 0; sc < S; ++sc) {
                            const long long mz = bz + 2 * sc;
                            const long long R = mxy + mz * mz;
                            if (R > a.Rh || R >= top || R < s_bnd[0]) continue;
                            int lo = 0, hi = a.A;
                            while (hi - lo > 1) {
                                const int mid = (lo + hi) >> 1;
                                if (s_bnd[mid] <= R) lo = mid;
                                else hi = mid;
                            }
                            a.gw[(long long)lo * a.W + w] += a.gtab[(R - 3) >> 3];
                        }
                    }
                }
            }
}

__global__ void __launch_bounds__(256) k_rgf_norm(int N, long long W, int A, const double* __restrict__ gw,
                                                  const double* __restrict__ I, double l3, int normalise,
                                                  double* scale, double* g0) {
    // block j: sum over the full grid = sum over the wedge with multiplicity
    // (number of distinct permutations) x prod over axes (1 at 0 and N/2, else 2)
    __shared__ double s_part[256];
    const int j = blockIdx.x;
    const int M = N / 2;
    double acc = 0.0;
    for (long long w = threadIdx.x; w < W; w += blockDim.x) {
        int a, b, c;
        wedge_decode(w, a, b, c);
        const int perms = (a == b && b == c) ? 1 : (a == b || b == c) ? 3 : 6;
        const double ax = (a == 0 || a == M) ? 1.0 : 2.0, bx = (b == 0 || b == M) ? 1.0 : 2.0,
                     cx = (c == 0 || c == M) ? 1.0 : 2.0;
        acc += perms * ax * bx * cx * gw[(long long)j * W + w];
    }
    s_part[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s_part[threadIdx.x] += s_part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // gw already carries the s^-3 sample weight (folded into the g table)
        const double sum = s_part[0];
        if (normalise && sum > 0.0) {
            scale[j] = I[j] / (l3 * sum);
            g0[j] = I[j] / l3;
        } else {
            scale[j] = 1.0;
            g0[j] = sum;
        }
    }
}


// One-shell table of the instantaneous field: sum_j Ghat_j per wedge row.
__global__ void __launch_bounds__(256) k_gsum(long long W, int A, int gstride, const float* __restrict__ ghat,
                                              const double* __restrict__ g0, float* __restrict__ gsum,
                                              double* __restrict__ g0sum) {
    const long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (w < W) {
        double s = 0.0;
        for (int j = 0; j < A; ++j) s += (double)ghat[w * gstride + j];
        gsum[8 * w] = (float)s;
        for (int c = 1; c < 8; ++c) gsum[8 * w + c] = 0.0f;
    }
    if (w == 0) {
        double d = 0.0;
        for (int j = 0; j < A; ++j) d += g0[j];
        *g0sum = d;
    }
}

__global__ void k_near_prep(const double* gw0, const double* scale0, double* gnear, double* g0_far) {
    // one thread: the near cube is (2R+1)^3 = 125 cells
    const int Wn = (kNearR + 1) * (kNearR + 2) * (kNearR + 3) / 6;
    for (int w = 0; w < Wn; ++w) gnear[w] = gw0[w] * (*scale0);
    gnear[Wn] = *scale0; // the shell's normalisation factor, for the sub-cell near field
    double sum = 0.0;
    for (int dx = -kNearR; dx <= kNearR; ++dx)
        for (int dy = -kNearR; dy <= kNearR; ++dy)
            for (int dz = -kNearR; dz <= kNearR; ++dz) sum += gnear[near_wedge(dx, dy, dz)];
    *g0_far -= sum;
}

__global__ void __launch_bounds__(256) k_near_scatter(NearScatter a, int N) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.n * kNearCube) return;
    near_scatter_item(a, N, idx);
}

__global__ void __launch_bounds__(256) k_near_fold(const long long* __restrict__ cell, const long long* __restrict__ q,
                                                   long long n, int N, double* __restrict__ acc, float* __restrict__ out,
                                                   long long* __restrict__ grid) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * kNearCube) return;
    const long long s = idx / kNearCube;
    const int m = (int)(idx % kNearCube);
    if (q[s] == 0) return;
    // the entry's own deposit cell (the cube's centre): the transforms have
    // read it, so it is cleared for the next deposit
    if (grid && m == kNearCube / 2) grid[cell[s]] = 0;
    int dx, dy, dz;
    const long long t = near_target(cell[s], m, N, dx, dy, dz);
    // the first thread to reach a cell takes its whole sum and clears it
    const double v = __longlong_as_double(
        (long long)atomicExch(reinterpret_cast<unsigned long long*>(acc + t), 0ULL));
    if (v != 0.0) out[t] = (float)((double)out[t] + v);
}

// Sub-cell near field (particle-mesh hybrid of the Discussion): one thread
// per (source, target cell of its near cube).  The target's value is the s^3
// sub-sample average of g around the source's own position, over the periodic
// images, inside the innermost shell [0, r_hi) and the horizon, times the
// shell's normalisation factor f0 and U S q.
//
// Everything per sample is FP32: the sample's offset from the source, r^2,
// the two factors of g that depend on r through the light-cone redshift
// z_s(r) from a table (linear in r), the kernel formula, and a compensated
// (Kahan) sum.  Only the shell and horizon test of
// a sample whose FP32 r^2 lies within `win2f` of rtop^2 is redone in FP64 from
// the FP64 sample position.  The FP32 sample coordinate is off by at most
// u (2 rtop + 5 l) per axis (u = 2^-24: the roundings of the image offset,
// of the sub-sample offset and of their sum, for an image with |c| < rtop +
// l/2 on every axis), so near the shell edge r^2 is off by at most
// u (10 rtop^2 + 18 rtop l); win2f = 1e-5 (rtop^2 + rtop l) is nine times
// that or more.
__device__ __forceinline__ void image_range(double b, double L, double invL, double reach, int U, int& lo, int& hi) {
    // images u with |b + u L| < reach (reach carries a relative margin)
    lo = (int)ceil((-reach - b) * invL);
    hi = (int)floor((reach - b) * invL);
    lo = lo < -U ? -U : lo;
    hi = hi > U ? U : hi;
}

__global__ void __launch_bounds__(256, 2) k_near_pm(NearPmArgs a, double* __restrict__ acc) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.n * kNearCube) return;
    const long long s = idx / kNearCube;
    const int m = (int)(idx % kNearCube);
    const long long qs = a.q[s];
    if (qs == 0) return;
    int dx, dy, dz;
    const long long t = near_target(a.cell[s], m, a.N, dx, dy, dz);
    const double l = a.l;
    // target cell centre minus source (central image)
    const double bx = l * dx - a.off[3 * s], by = l * dy - a.off[3 * s + 1], bz = l * dz - a.off[3 * s + 2];
    const int S = a.S;
    // an image contributes only if on every axis its cell centre lies within
    // rtop + l/2 of the source (every sample is within l/2 of the centre)
    const double reach = (a.rtop + 0.5 * l) * (1.0 + 1e-6) + 1e-6 * l;
    const double invL = 1.0 / a.L;
    int ulo, uhi, vlo, vhi, wlo, whi;
    image_range(bx, a.L, invL, reach, a.U, ulo, uhi);
    image_range(by, a.L, invL, reach, a.U, vlo, vhi);
    image_range(bz, a.L, invL, reach, a.U, wlo, whi);
    const float inv_h = (float)((a.K - 1) / a.rtop);
    const float xcut = a.xcut; // Eq. 15's cut r = 97.39 alpha as r / (116.29 alpha); none for the rough horizon
    const float lf = (float)l;
    const float invS = 1.0f / (float)S;
    const float rtop2f = a.rtop2f, win2f = a.win2f;
    float sum = 0.0f, comp = 0.0f; // Kahan
    for (int u = ulo; u <= uhi; ++u)
        for (int v = vlo; v <= vhi; ++v)
            for (int w = wlo; w <= whi; ++w) {
                const double cx = bx + u * a.L, cy = by + v * a.L, cz = bz + w * a.L;
                const float cxf = (float)cx, cyf = (float)cy, czf = (float)cz;
                // no sample of this image's target cell can reach the shell:
                // |c| >= rtop + half-diagonal, with a relative margin
                if (cxf * cxf + cyf * cyf + czf * czf > a.prune2f) continue;
                for (int ia = 0; ia < S; ++ia) {
                    const float px = cxf + lf * (((float)ia + 0.5f) * invS - 0.5f);
                    for (int ib = 0; ib < S; ++ib) {
                        const float py = cyf + lf * (((float)ib + 0.5f) * invS - 0.5f);
                        const float rxy2 = px * px + py * py;
                        if (rxy2 > rtop2f + win2f) continue; // every sample of the row is outside
                        for (int ic = 0; ic < S; ++ic) {
                            const float pz = czf + lf * (((float)ic + 0.5f) * invS - 0.5f);
                            const float r2 = rxy2 + pz * pz;
                            bool in = r2 < rtop2f;
                            if (fabsf(r2 - rtop2f) <= win2f) {
                                // too close to call in FP32: decide in FP64
                                const double qx = cx + l * ((ia + 0.5) / S - 0.5), qy = cy + l * ((ib + 0.5) / S - 0.5),
                                             qz = cz + l * ((ic + 0.5) / S - 0.5);
                                const double r = sqrt(qx * qx + qy * qy + qz * qz);
                                in = r < a.rhi && r <= a.rh;
                            }
                            if (!in) continue;
                            const float r = sqrtf(r2);
                            const float xt = r * inv_h;
                            int k0 = (int)xt;
                            if (k0 > a.K - 2) k0 = a.K - 2;
                            const float fr = xt - (float)k0;
                            const float2 t0 = __ldg(a.tab + k0), t1 = __ldg(a.tab + k0 + 1);
                            const float hz = t0.x + fr * (t1.x - t0.x); // (1+z_obs)^3 / ((4 pi)^2 (1+z_s))
                            float f;
                            if (a.kind == 1) {
                                f = r < a.kmax ? expf(-r * a.inv_klen) : 0.0f;
                            } else {
                                const float x = r * (t0.y + fr * (t1.y - t0.y)); // r / (116.29 alpha(z_s))
                                // f_mod of Eq. 15 with x^0.68 = 2^(0.68 log2 x), clamped at 0
                                // (only the rough horizon reaches where it turns negative)
                                f = x > xcut ? 0.0f : fmaxf(1.7f * expf(-exp2f(0.68f * log2f(x))) - 0.7f, 0.0f);
                            }
                            if (f == 0.0f) continue;
                            const float y = __fdividef(hz * f, r2) - comp;
                            const float tt = sum + y;
                            comp = (tt - sum) - y;
                            sum = tt;
                        }
                    }
                }
            }
    const double tot = (double)sum - (double)comp;
    if (tot != 0.0) atomicAdd(acc + t, a.U_out * a.slot_S[a.slot] * (double)qs * a.f0[0] * tot / ((double)S * S * S));
}

} // namespace

void launch_near_pm(const NearPmArgs& a, double* acc, cudaStream_t st) {
    const long long total = a.n * kNearCube;
    if (total <= 0) return;
    launch_k(k_near_pm, (unsigned)((total + 255) / 256), 256, 0, st, a, acc);
}

void launch_gsum(long long W, int A, int gstride, const float* ghat, const double* g0, float* gsum, double* g0sum,
                 cudaStream_t st) {
    if (W <= 0) return;
    const long long blocks = (W + 255) / 256;
    k_gsum<<<(unsigned)blocks, 256, 0, st>>>(W, A, gstride, ghat, g0, gsum, g0sum);
}

void launch_near_prep(const double* gw0, const double* scale0, double* gnear, double* g0_far, cudaStream_t st) {
    k_near_prep<<<1, 1, 0, st>>>(gw0, scale0, gnear, g0_far);
}

void launch_near_scatter(const NearScatter& a, int N, cudaStream_t st) {
    const long long total = a.n * kNearCube;
    if (total <= 0) return;
    launch_k(k_near_scatter, (unsigned)((total + 255) / 256), 256, 0, st, a, N);
}

void launch_near_fold(const long long* cell, const long long* q, long long n, int N, double* acc, float* out,
                      long long* grid, cudaStream_t st) {
    const long long total = n * kNearCube;
    if (total <= 0) return;
    launch_k(k_near_fold, (unsigned)((total + 255) / 256), 256, 0, st, cell, q, n, N, acc, out, grid);
}

// Zero the deposit cells of a near-field list (entries with a non-zero share).
__global__ void __launch_bounds__(256) k_cells_clear(const long long* __restrict__ cell,
                                                     const long long* __restrict__ q, long long n,
                                                     long long* __restrict__ grid) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && q[i] != 0) grid[cell[i]] = 0;
}

void launch_cells_clear(const long long* cell, const long long* q, long long n, long long* grid, cudaStream_t st) {
    if (n <= 0) return;
    launch_k(k_cells_clear, (unsigned)((n + 255) / 256), 256, 0, st, cell, q, n, grid);
}

void launch_src_prep(const double* pos, const double* lum, long long n, unsigned long long* maxbits, int* err,
                     SlotMeta m, cudaStream_t st) {
    launch_k(k_src_prep, 1, kPrepThreads, 0, st, pos, lum, n, maxbits, err, m);
}

void launch_deposit(const double* pos, const double* lum, long long n, int N, double l, int deposit,
                    const unsigned long long* maxbits, long long* grid, SlotMeta m, int* err, cudaStream_t st,
                    long long* cell_out, long long* q_out, double* off_out) {
    // one source per thread, in blocks of 32 to 256 threads chosen so that
    // the sources spread over about two CTAs per SM: each costs a few FP64
    // divisions, and FP64 issue per SM is narrow on this GPU
    const long long per_cta = (n + 2 * 152 - 1) / (2 * 152);
    const int tb = (int)(per_cta <= 32 ? 32 : per_cta >= 256 ? 256 : (per_cta + 31) / 32 * 32);
    const long long blocks = n > 0 ? (n + tb - 1) / tb : 1;
    if (deposit == LC_DEPOSIT_CIC)
        launch_k(k_deposit<1>, (unsigned)blocks, tb, 0, st, pos, lum, n, N, l, maxbits, grid, m, err, cell_out, q_out,
                 (double*)nullptr);
    else
        launch_k(k_deposit<0>, (unsigned)blocks, tb, 0, st, pos, lum, n, N, l, maxbits, grid, m, err, cell_out, q_out,
                 off_out);
}

// f_diff = (J_instant - J) / J, the difference taken and divided in FP64 and
// rounded once; 0 where both fields are 0 (IEEE +-inf where only J is 0)
__global__ void __launch_bounds__(256) k_fdiff(long long n, const float* __restrict__ j,
                                               const float* __restrict__ ji, float* __restrict__ out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double a = j[i], b = ji[i];
        out[i] = (a == 0.0 && b == 0.0) ? 0.0f : (float)((b - a) / a);
    }
}

// Device -> page-locked host copy by the SMs (16-byte stores through the
// host mapping of the buffer), for the waiting host output path.
__global__ void __launch_bounds__(256) k_copy_out(long long n4, const float4* __restrict__ src, float4* dst) {
    // four loads in flight per thread before the stores (a small grid copies
    // at the host link's rate only with enough bytes outstanding)
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n4; i += 4 * stride) {
        float4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = src[i + u * stride];
#pragma unroll
        for (int u = 0; u < 4; ++u) dst[i + u * stride] = v[u];
    }
    for (; i < n4; i += stride) dst[i] = src[i];
}

void launch_copy_out(long long n4, const float4* src, float4* dst, int ctas, cudaStream_t st) {
    if (n4 <= 0) return;
    const long long need = (n4 + 255) / 256;
    k_copy_out<<<(unsigned)(need < ctas ? need : ctas), 256, 0, st>>>(n4, src, dst);
}

void launch_fdiff(long long n, const float* j, const float* j_inst, float* out, cudaStream_t st) {
    if (n <= 0) return;
    const long long blocks = (n + 255) / 256;
    k_fdiff<<<(unsigned)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, st>>>(n, j, j_inst, out);
}

void launch_rgf_accum(const RgfAccumArgs& a, cudaStream_t st) {
    if (a.W <= 0) return;
    k_rgf_accum<<<(unsigned)((a.W + 127) / 128), 128, 0, st>>>(a);
}

void launch_rgf_norm(int N, long long W, int A, const double* gw, const double* I, double l3, int normalise,
                     double* scale, double* g0, cudaStream_t st) {
    k_rgf_norm<<<A, 256, 0, st>>>(N, W, A, gw, I, l3, normalise, scale, g0);
}

} // namespace lc
