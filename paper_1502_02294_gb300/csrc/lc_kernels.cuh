// lc_kernels.cuh -- the per-grid-size FFT pass kernels of the retarded-field
// path (templated on N, instantiated once per supported N).
//
//  k_rows_r2c : z-axis real->complex rows (Eq. 12 forward), prologue reads the
//               int64 fixed-point deposit grid (source term f_n, Eq. 11), a
//               float grid, or gathers a Green's function from its wedge.
//  k_cols     : y- or x-axis complex pass over 16-column tiles.  Fused modes:
//                 forward x-pass epilogue -> history ring slot (FP32 / BF16),
//                 forward x-pass epilogue -> real part on the symmetric wedge
//                   (the stored Ghat_n of step 3, Section 2.2),
//                 inverse x-pass prologue -> the shell multiply-accumulate
//                   Jhat(k) = sum_n Ghat_n(k) fhat_{s-n}(k)  (Eq. 13 summed
//                   over slices, steps 5-6) with the k = 0 mode overwritten
//                   by its FP64 value.
//  k_rows_c2r : z-axis complex->real rows (Eq. 12 inverse) with the output
//               scale U / N^3 fused.
#pragma once
#include "lc_fft.cuh"

namespace lc {

enum { ROW_IN_I64 = 0, ROW_IN_F32 = 1, ROW_IN_WEDGE = 2 };
// COL_IN_MAC_*_X: the shell MAC whose newest slice (lookback 0) is this
// tile of the y-transformed spectrum `src`, forward x-transformed in the
// same kernel and written to its ring slot (`ring_out`, slot `wslot`) on the
// way, with the arithmetic of the plain x pass into the ring
enum { COL_IN_PLAIN = 0, COL_IN_MAC_F32 = 1, COL_IN_MAC_BF16 = 2, COL_IN_MAC_F32_X = 3, COL_IN_MAC_BF16_X = 4 };
// COL_OUT_BF16 / COL_OUT_RING_F32 write one slot of the history ring, whose
// layout is [tile][slot][N x CW elements]: the history of an x-pass tile over
// all slots is one contiguous run, read as a stream by the shell MAC
enum { COL_OUT_PLAIN = 0, COL_OUT_BF16 = 1, COL_OUT_WEDGE = 2, COL_OUT_RING_F32 = 3 };

struct RowR2CArgs {
    int in_mode;
    long long nrows;
    const long long* grid;    // ROW_IN_I64: N^3 int64
    const double* slot_S;     // ROW_IN_I64: fixed-point unit of the slot
    const long long* slot_total;
    int slot;
    int bf16;                 // ROW_IN_I64: 1 -> values / (S * total), else * S
    int zero_in;              // ROW_IN_I64: leave the grid all zero for the next deposit
    // ROW_IN_I64, optional (nullptr: every row read): per row (x N + y) the
    // push counter of its last deposit, and the counter (*stamp); a row whose
    // value differs holds no share of this push and is all zero, so the lanes
    // forms of the z pass skip its loads and transform (its half spectrum is 0)
    const unsigned* rowstamp;
    const unsigned* stamp;
    const float* fin;         // ROW_IN_F32
    const double* gw;         // ROW_IN_WEDGE: wedge values of one shell (FP64)
    const double* gscale;     // ROW_IN_WEDGE: that shell's normalisation factor
    int near_r;               // ROW_IN_WEDGE: displacements with all |folded| <= near_r read as 0 (-1: none)
    float2* dst;              // half spectrum, rows of NRP
    const float2* tw;
};

struct ColArgs {
    int axis;                 // 0: y-pass, 1: x-pass
    int in_mode, out_mode, dir;
    const float2* src;
    float2* dst;
    __nv_bfloat162* dst_bf16;
    // shell MAC (inverse x-pass); the ring is [tile][slot][tile elements]
    const void* ring;
    long long slot_elems;     // complex elements per ring slot (N^2 (N/2 + 1))
    int n_ring, step, A;
    int wslot;                // ring write: the slot being written
    const int* slot_step;
    const double* slot_S;
    const long long* slot_total;
    const float* ghat;        // [wedge][A] real Ghat of this step
    const double* g0;         // [A] FP64 Ghat_j(0)
    int gstride;              // row stride of the Ghat table (A rounded up to 8)
    int instant;              // 1: every shell uses the observing step's slice (Eq. 18)
    int tile0;                // first tile of this launch (tiles before it are skipped)
    void* ring_out;           // COL_IN_MAC_*_X: the ring the newest slice is written to
    // wedge extract (forward x-pass of a Green's function)
    float* wedge_out;
    int wedge_A, wedge_j;     // wedge_A: row stride of the table written
    const float2* tw;
    // tensor map of `src` seen as [p][q][2 NRP floats] with the box of this
    // pass's axis (TMA column passes; null: none made for this buffer), and
    // the error word a timed-out copy wait reports to (may be null)
    const CUtensorMap* tmap;
    int* err;
};

struct RowC2RArgs {
    long long nrows;
    const float2* src;
    float* out;
    float scale;
    const float2* tw;
    // plane kernels: the near-field list, run by near.ctas CTAs launched
    // after the N plane CTAs, on SMs the planes leave idle (0: none)
    NearScatter near;
};

// The CTAs of a plane kernel from block FIRST on (past its planes) walk the
// near-field list of the N^3 grid.
template <int N, int NT, int FIRST = N>
__device__ __forceinline__ void plane_near_ctas(const NearScatter& a) {
    const long long total = a.n * kNearCube;
    for (long long i = (long long)(blockIdx.x - FIRST) * NT + threadIdx.x; i < total; i += (long long)a.ctas * NT)
        near_scatter_item(a, N, i);
}

constexpr int kMaxShells = 1024;

// The ring slots that hold the active slices of a step, compacted in
// increasing lookback j: slot, j, scale D (the slot's luminosity total for
// BF16 history, 1 for FP32) and the FP64 k = 0 sum  sum_j Ghat_j(0) S_j q_j.
// Run by one whole warp: 32 slices per round trip to memory.
// instant != 0: every shell reads the slice of the observing step itself
// (the source frozen at the observing redshift, Eq. 18).
__device__ __forceinline__ void mac_slot_list(int A, int step, int n_ring, const int* slot_step,
                                              const long long* slot_total, const double* slot_S, const double* g0,
                                              bool bf16, int* out_slot, int* out_j, float* out_D, int* nv_out,
                                              double* dc_out, int instant = 0) {
    const int lane = threadIdx.x & 31;
    int nv = 0;
    double dc = 0.0;
    for (int j0 = 0; j0 < A; j0 += 32) {
        const int j = j0 + lane;
        const int n = instant ? step : step - j;
        bool valid = false;
        int slot = 0;
        double lum = 0.0;
        if (j < A && n >= 0) {
            slot = n % n_ring;
            if (slot_step[slot] == n) {
                const long long tot = slot_total[slot];
                if (tot != 0) {
                    valid = true;
                    lum = slot_S[slot] * (double)tot;
                }
            }
        }
        const unsigned ball = __ballot_sync(0xffffffffu, valid);
        const int pos = nv + __popc(ball & ((1u << lane) - 1u));
        double part = 0.0;
        if (valid) {
            out_slot[pos] = slot;
            out_j[pos] = j;
            out_D[pos] = bf16 ? (float)lum : 1.0f;
            part = g0[j] * lum;
        }
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        dc += part;
        nv += __popc(ball);
    }
    if (lane == 0) {
        *nv_out = nv;
        *dc_out = dc;
    }
}

template <int N> __host__ __device__ constexpr size_t rows_smem_bytes() {
    return sizeof(float2) * (N + (size_t)N * odd_pad(row_pairs_of(N)));
}
template <int N> __host__ __device__ constexpr size_t cols_smem_bytes() {
    // twiddles + the padded tile + the compact shell list (offset, lookback, scale, slot)
    return sizeof(float2) * (N + (size_t)N * odd_pad(cw_of(N))) + (size_t)kMaxShells * 20 + 16;
}

// ------------------------------------------------------------------------
// z rows, real -> complex, persistent: a CTA owns row blocks blockIdx.x,
// +gridDim.x, ...; every thread issues all global loads of the next block
// (compile-time count, registers) before transforming the current one.
template <int N, int IN>
__global__ void __launch_bounds__(kThreads) k_rows_r2c(RowR2CArgs a, int nblocks) {
    constexpr int B = row_pairs_of(N), BP = odd_pad(B), NRP = nrp_of(N), H = N / 2 + 1;
    constexpr int TILE = 2 * B * N, PER = (TILE + kThreads - 1) / kThreads;
    extern __shared__ float4 smem_raw[];
    float2* tw = reinterpret_cast<float2*>(smem_raw);
    float2* buf = tw + N;
    float scale = 1.0f;
    double gsc = 1.0;
    if constexpr (IN == ROW_IN_I64) {
        const double S = a.slot_S[a.slot];
        const long long tot = a.slot_total[a.slot];
        // FP32 history: luminosity units (S is a power of two: exact);
        // BF16 history: divided by the total so that |fhat| <= 1.
        scale = a.bf16 ? (tot > 0 ? (float)(1.0 / (double)tot) : 0.0f) : (float)S;
    }
    if constexpr (IN == ROW_IN_WEDGE) gsc = *a.gscale;
    auto fetch = [&](int blk, float* val) {
        const long long row0 = (long long)blk * (2 * B);
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int idx = threadIdx.x + i * kThreads;
            const int rr = idx / N, t = idx % N;
            const long long grow = row0 + rr;
            val[i] = 0.0f;
            if ((TILE % kThreads == 0 || idx < TILE) && grow < a.nrows) {
                if constexpr (IN == ROW_IN_I64) val[i] = __ll2float_rn(a.grid[grow * N + t]) * scale;
                else if constexpr (IN == ROW_IN_F32) val[i] = a.fin[grow * N + t];
                else {
                    const int x = (int)(grow / N), y = (int)(grow % N);
                    const int fx = x <= N - x ? x : N - x, fy = y <= N - y ? y : N - y, fz = t <= N - t ? t : N - t;
                    const int mx = fx > fy ? (fx > fz ? fx : fz) : (fy > fz ? fy : fz);
                    val[i] = mx <= a.near_r ? 0.0f : (float)(a.gw[wedge_of(x, y, t, N)] * gsc);
                }
            }
        }
    };
    for (int i = threadIdx.x; i < N; i += kThreads) tw[i] = a.tw[i];
    float cur[PER], nxt[PER];
    int blk = blockIdx.x;
    if (blk < nblocks) fetch(blk, cur);
    float* bf = reinterpret_cast<float*>(buf);
    while (blk < nblocks) {
        const int next = blk + gridDim.x;
        if (next < nblocks) fetch(next, nxt);
        __syncthreads(); // the previous block has left shared memory
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int idx = threadIdx.x + i * kThreads;
            if (TILE % kThreads == 0 || idx < TILE) {
                const int rr = idx / N, t = idx % N;
                bf[2 * (t * BP + (rr >> 1)) + (rr & 1)] = cur[i];
            }
        }
        __syncthreads();
        fft_smem<N, -1, B, BP>(buf, tw);
        // unpack the two real rows of each pair: X_a = (Z_k + conj Z_{N-k}) / 2,
        // X_b = (Z_k - conj Z_{N-k}) / (2i)
        const long long row0 = (long long)blk * (2 * B);
        for (int idx = threadIdx.x; idx < 2 * B * H; idx += kThreads) {
            const int rr = idx / H, k = idx % H;
            const long long grow = row0 + rr;
            if (grow >= a.nrows) continue;
            const int pair = rr >> 1;
            const float2 zk = buf[k * BP + pair];
            const float2 zn = buf[(k == 0 ? 0 : N - k) * BP + pair];
            float2 x;
            if ((rr & 1) == 0) x = make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
            else x = make_float2(0.5f * (zk.y + zn.y), 0.5f * (zn.x - zk.x));
            a.dst[grow * NRP + k] = x;
        }
#pragma unroll
        for (int i = 0; i < PER; ++i) cur[i] = nxt[i];
        blk = next;
    }
}

// ------------------------------------------------------------------------
// y or x pass over one N x CW tile (CW consecutive r-columns of one line, or
// CW Nyquist columns of CW lines).  NT = N * CW / 8 threads, 8 elements each.
template <int N, int DIR, int IN, int OUT>
__global__ void __launch_bounds__(col_threads_of(N)) k_cols(ColArgs a) {
    constexpr bool BFR = IN == COL_IN_MAC_BF16 || IN == COL_IN_MAC_BF16_X; // BF16 ring
    constexpr bool FWDX = IN == COL_IN_MAC_F32_X || IN == COL_IN_MAC_BF16_X;
    constexpr int NT = col_threads_of(N);
    constexpr int CW = cw_of(N), BP = odd_pad(CW), NRP = nrp_of(N), M = N / 2, NCH = M / CW;
    constexpr int TILE = N * CW, PER = (TILE + NT - 1) / NT;
    constexpr long long PLANE = (long long)N * NRP;
    extern __shared__ float4 smem_raw[];
    float2* tw = reinterpret_cast<float2*>(smem_raw);
    float2* buf = tw + N;
    long long* s_off = reinterpret_cast<long long*>(buf + N * BP);
    int* s_j = reinterpret_cast<int*>(s_off + kMaxShells);
    float* s_D = reinterpret_cast<float*>(s_j + kMaxShells);
    __shared__ int s_nv;
    __shared__ double s_dc;

    const int tile = blockIdx.x + a.tile0;
    const bool nyq = tile >= N * NCH;
    int line = 0, chunk = 0;
    long long base, ts, cs;
    if (!nyq) {
        line = tile / NCH;
        chunk = tile % NCH;
        if (a.axis == 0) { base = line * PLANE + chunk * CW; ts = NRP; cs = 1; }
        else { base = (long long)line * NRP + chunk * CW; ts = PLANE; cs = 1; }
    } else {
        line = (tile - N * NCH) * CW; // first of CW lines, column r = N/2
        if (a.axis == 0) { base = line * PLANE + M; ts = NRP; cs = PLANE; }
        else { base = (long long)line * NRP + M; ts = PLANE; cs = NRP; }
    }
    long long addr[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int idx = threadIdx.x + i * NT;
        addr[i] = base + (long long)(idx / CW) * ts + (idx % CW) * cs;
    }
    float2 val[PER];

    if constexpr (IN == COL_IN_PLAIN) {
#pragma unroll
        for (int i = 0; i < PER; ++i)
            if (TILE % NT == 0 || threadIdx.x + i * NT < TILE) val[i] = a.src[addr[i]];
        for (int i = threadIdx.x; i < N; i += NT) tw[i] = a.tw[i];
    } else {
        // compact list of the ring slots that hold the slices of this step
        const bool dc_tile = (a.axis == 1) && !nyq && line == 0 && chunk == 0;
        int* s_slot = reinterpret_cast<int*>(s_D + kMaxShells);
        if (threadIdx.x < 32)
            mac_slot_list(a.A, a.step, a.n_ring, a.slot_step, a.slot_total, a.slot_S, a.g0, BFR, s_slot, s_j, s_D,
                          &s_nv, &s_dc, a.instant);
        __syncthreads();
        for (int v = threadIdx.x; v < s_nv; v += NT) s_off[v] = (long long)s_slot[v] * TILE;
        for (int i = threadIdx.x; i < N; i += NT) tw[i] = a.tw[i];
        // wedge rows of Ghat for this thread's elements (x pass: t runs over p)
        const float* g[PER];
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int idx = threadIdx.x + i * NT;
            const int t = idx / CW, col = idx % CW;
            const int q = nyq ? line + col : line;
            const int r = nyq ? M : chunk * CW + col;
            g[i] = a.ghat + wedge_of(t, q, r, N) * a.gstride;
            val[i] = make_float2(0.f, 0.f);
        }
        __syncthreads();
        float2 fx[FWDX ? PER : 1];
        if constexpr (FWDX) {
            // the newest slice: the forward x transform of this tile of
            // `src`, stored to its ring slot exactly as the plain x pass
            // into the ring stores it, and kept in registers for lookback 0
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int idx = threadIdx.x + i * NT;
                if (TILE % NT == 0 || idx < TILE) buf[(idx / CW) * BP + (idx % CW)] = a.src[addr[i]];
            }
            __syncthreads();
            fft_smem<N, -1, CW, BP, NT>(buf, tw);
            const long long wbase = ((long long)tile * a.n_ring + a.wslot) * TILE;
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int idx = threadIdx.x + i * NT;
                fx[i] = make_float2(0.f, 0.f);
                if (TILE % NT == 0 || idx < TILE) {
                    const float2 v = buf[(idx / CW) * BP + (idx % CW)];
                    if constexpr (BFR) {
                        const __nv_bfloat162 b = __floats2bfloat162_rn(v.x, v.y);
                        reinterpret_cast<__nv_bfloat162*>(a.ring_out)[wbase + idx] = b;
                        fx[i] = __bfloat1622float2(b);
                    } else {
                        reinterpret_cast<float2*>(a.ring_out)[wbase + idx] = v;
                        fx[i] = v;
                    }
                }
            }
            __syncthreads(); // buf is free again for the inverse transform
        }
        const int nv = s_nv;
        const long long tbase = (long long)tile * a.n_ring * TILE;
        // shells outer, the tile's elements inner: PER independent ring loads
        // (and Ghat loads) in flight per thread per shell, and the next
        // shell's loads issued before this shell's FMAs (same order of sums)
        auto fetch = [&](int v, float2 (&f)[PER], float (&gv)[PER]) {
            const long long off = s_off[v];
            const int jv = s_j[v];
            const bool own = FWDX && jv == 0; // the newest slice, already in registers
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                if (TILE % NT == 0 || threadIdx.x + i * NT < TILE) {
                    const long long ri = off + tbase + threadIdx.x + i * NT; // tile-major ring slot
                    if (own) f[i] = fx[FWDX ? i : 0];
                    else if constexpr (!BFR) f[i] = reinterpret_cast<const float2*>(a.ring)[ri];
                    else f[i] = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(a.ring)[ri]);
                    gv[i] = __ldg(g[i] + jv);
                } else {
                    f[i] = make_float2(0.f, 0.f);
                    gv[i] = 0.f;
                }
            }
        };
        float2 f[PER], fn[PER];
        float gv[PER], gn[PER];
        if (nv > 0) fetch(0, f, gv);
        for (int v = 0; v < nv; ++v) {
            if (v + 1 < nv) fetch(v + 1, fn, gn);
            const float D = s_D[v];
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const float w = gv[i] * D;
                val[i].x = fmaf(w, f[i].x, val[i].x);
                val[i].y = fmaf(w, f[i].y, val[i].y);
            }
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                f[i] = fn[i];
                gv[i] = gn[i];
            }
        }
        if (dc_tile && threadIdx.x == 0) val[0] = make_float2((float)s_dc, 0.0f);
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int idx = threadIdx.x + i * NT;
        if (TILE % NT == 0 || idx < TILE) buf[(idx / CW) * BP + (idx % CW)] = val[i];
    }
    __syncthreads();
    fft_smem<N, DIR, CW, BP, NT>(buf, tw);
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int idx = threadIdx.x + i * NT;
        if (!(TILE % NT == 0 || idx < TILE)) continue;
        const int t = idx / CW, col = idx % CW;
        const float2 v = buf[t * BP + col];
        if constexpr (OUT == COL_OUT_PLAIN) {
            a.dst[addr[i]] = v;
        } else if constexpr (OUT == COL_OUT_BF16) {
            a.dst_bf16[addr[i]] = __floats2bfloat162_rn(v.x, v.y);
        } else {
            const int q = nyq ? line + col : line;
            const int r = nyq ? M : chunk * CW + col;
            if (t <= q && q <= r) a.wedge_out[wedge_index(t, q, r) * a.wedge_A + a.wedge_j] = v.x;
        }
    }
}

// ------------------------------------------------------------------------
// Plain y / x pass, persistent: each CTA walks tiles blockIdx.x, +gridDim.x,
// ... and issues the next tile's global loads (into registers) before it
// transforms and stores the current one, so loads stay in flight while the
// shared-memory FFT runs.
template <int N> struct ColGeom {
    static constexpr int CW = cw_of(N), NRP = nrp_of(N), M = N / 2, NCH = M / CW;
    static constexpr long long PLANE = (long long)N * NRP;
    long long base, ts, cs;
    int line, chunk;
    bool nyq;
    __device__ __forceinline__ ColGeom(int tile, int axis) {
        nyq = tile >= N * NCH;
        if (!nyq) {
            line = tile / NCH;
            chunk = tile % NCH;
            if (axis == 0) { base = line * PLANE + chunk * CW; ts = NRP; cs = 1; }
            else { base = (long long)line * NRP + chunk * CW; ts = PLANE; cs = 1; }
        } else {
            line = (tile - N * NCH) * CW;
            chunk = 0;
            if (axis == 0) { base = line * PLANE + M; ts = NRP; cs = PLANE; }
            else { base = (long long)line * NRP + M; ts = PLANE; cs = NRP; }
        }
    }
    __device__ __forceinline__ long long at(int idx) const { return base + (long long)(idx / CW) * ts + (idx % CW) * cs; }
};

template <int N, int DIR, int OUT>
__global__ void __launch_bounds__(col_threads_of(N)) k_cols_pp(ColArgs a, int ntiles) {
    constexpr int NT = col_threads_of(N);
    constexpr int CW = cw_of(N), BP = odd_pad(CW), M = N / 2;
    constexpr int TILE = N * CW, PER = (TILE + NT - 1) / NT;
    extern __shared__ float4 smem_raw[];
    float2* tw = reinterpret_cast<float2*>(smem_raw);
    float2* buf = tw + N;
    for (int i = threadIdx.x; i < N; i += NT) tw[i] = a.tw[i];
    int tile = blockIdx.x;
    float2 cur[PER];
    if (tile < ntiles) {
        const ColGeom<N> g(tile + a.tile0, a.axis);
#pragma unroll
        for (int i = 0; i < PER; ++i)
            if (TILE % NT == 0 || threadIdx.x + i * NT < TILE) cur[i] = a.src[g.at(threadIdx.x + i * NT)];
    }
    while (tile < ntiles) {
        const ColGeom<N> g(tile + a.tile0, a.axis);
        const int next = tile + gridDim.x;
        float2 nxt[PER];
        if (next < ntiles) {
            const ColGeom<N> gn(next + a.tile0, a.axis);
#pragma unroll
            for (int i = 0; i < PER; ++i)
                if (TILE % NT == 0 || threadIdx.x + i * NT < TILE) nxt[i] = a.src[gn.at(threadIdx.x + i * NT)];
        }
        __syncthreads(); // the previous tile's results have left shared memory
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int idx = threadIdx.x + i * NT;
            if (TILE % NT == 0 || idx < TILE) buf[(idx / CW) * BP + (idx % CW)] = cur[i];
        }
        __syncthreads();
        fft_smem<N, DIR, CW, BP, NT>(buf, tw);
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int idx = threadIdx.x + i * NT;
            if (!(TILE % NT == 0 || idx < TILE)) continue;
            const int t = idx / CW, col = idx % CW;
            const float2 v = buf[t * BP + col];
            if constexpr (OUT == COL_OUT_PLAIN) {
                a.dst[g.at(idx)] = v;
            } else if constexpr (OUT == COL_OUT_BF16) {
                a.dst_bf16[((long long)(tile + a.tile0) * a.n_ring + a.wslot) * TILE + idx] =
                    __floats2bfloat162_rn(v.x, v.y);
            } else if constexpr (OUT == COL_OUT_RING_F32) {
                a.dst[((long long)(tile + a.tile0) * a.n_ring + a.wslot) * TILE + idx] = v;
            } else {
                const int q = g.nyq ? g.line + col : g.line;
                const int r = g.nyq ? M : g.chunk * CW + col;
                if (t <= q && q <= r) a.wedge_out[wedge_index(t, q, r) * a.wedge_A + a.wedge_j] = v.x;
            }
        }
#pragma unroll
        for (int i = 0; i < PER; ++i) cur[i] = nxt[i];
        tile = next;
    }
}

// Asynchronous global -> shared copies (LDGSTS) for the pipelined passes.
__device__ __forceinline__ void ldgsts16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(reinterpret_cast<unsigned long long>(src))
                 : "memory");
}
__device__ __forceinline__ void ldgsts8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(reinterpret_cast<unsigned long long>(src))
                 : "memory");
}
__device__ __forceinline__ void ldgsts_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int PENDING> __device__ __forceinline__ void ldgsts_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory");
}

// The pipelined plain pass (N >= 256): threads (8 elements each) and stages
// of tiles per CTA, one CTA per SM (measured at 256^3 against 6 stages, and
// against 3 stages with two CTAs of 256 threads per SM: both slower)
__host__ __device__ constexpr int cols_pl_threads(int n) { return col_threads_of(n); }
__host__ __device__ constexpr int cols_pl_stages(int n) { return 4; }
template <int N> __host__ __device__ constexpr size_t cols_pl_smem_bytes() {
    return sizeof(float2) * ((size_t)N + (size_t)cols_pl_stages(N) * N * cw_of(N));
}

// The pipelined persistent plain pass: tiles blockIdx.x, +gridDim.x, ... each copied
// straight into one of S shared-memory stages (16-byte asynchronous copies,
// 8-byte ones for the strided Nyquist tiles), S - 1 tiles in flight while
// one is transformed in place ([N][CW] rows: a half-warp reads one row of
// 16 complex or two of 8, so the dense layout is free of bank conflicts).
template <int N, int DIR, int OUT>
__global__ void __launch_bounds__(cols_pl_threads(N)) k_cols_pl(ColArgs a, int ntiles) {
    constexpr int NT = cols_pl_threads(N);
    constexpr int CW = cw_of(N), M = N / 2, S = cols_pl_stages(N);
    constexpr int TILE = N * CW;
    static_assert(CW % 2 == 0, "16-byte copies take two columns");
    extern __shared__ float4 smem_raw[];
    float2* tw = reinterpret_cast<float2*>(smem_raw);
    float2* stages = tw + N; // 16-byte aligned: N is even
    for (int i = threadIdx.x; i < N; i += NT) tw[i] = a.tw[i];
    auto load = [&](int tile, float2* dst) {
        const ColGeom<N> g(tile + a.tile0, a.axis);
        if (!g.nyq) {
            for (int c = threadIdx.x; c < TILE / 2; c += NT) ldgsts16(dst + 2 * c, a.src + g.at(2 * c));
        } else {
            for (int i = threadIdx.x; i < TILE; i += NT) ldgsts8(dst + i, a.src + g.at(i));
        }
    };
#pragma unroll
    for (int k = 0; k < S - 1; ++k) {
        const int t = blockIdx.x + k * gridDim.x;
        if (t < ntiles) load(t, stages + k * TILE);
        ldgsts_commit();
    }
    for (int k = 0;; ++k) {
        const int tile = blockIdx.x + k * gridDim.x;
        if (tile >= ntiles) break;
        // refill the stage that tile k - 1 used (its outputs are written)
        const int nt = blockIdx.x + (k + S - 1) * gridDim.x;
        if (nt < ntiles) load(nt, stages + ((k + S - 1) % S) * TILE);
        ldgsts_commit();
        ldgsts_wait<S - 1>(); // this thread's copies of tile k have landed
        __syncthreads();      // and everyone else's
        float2* buf = stages + (k % S) * TILE;
        fft_smem<N, DIR, CW, CW, NT>(buf, tw);
        const ColGeom<N> g(tile + a.tile0, a.axis);
        for (int idx = threadIdx.x; idx < TILE; idx += NT) {
            const int t = idx / CW, col = idx % CW;
            const float2 v = buf[idx];
            if constexpr (OUT == COL_OUT_PLAIN) {
                a.dst[g.at(idx)] = v;
            } else if constexpr (OUT == COL_OUT_BF16) {
                a.dst_bf16[((long long)(tile + a.tile0) * a.n_ring + a.wslot) * TILE + idx] =
                    __floats2bfloat162_rn(v.x, v.y);
            } else if constexpr (OUT == COL_OUT_RING_F32) {
                a.dst[((long long)(tile + a.tile0) * a.n_ring + a.wslot) * TILE + idx] = v;
            } else {
                const int q = g.nyq ? g.line + col : g.line;
                const int r = g.nyq ? M : g.chunk * CW + col;
                if (t <= q && q <= r) a.wedge_out[wedge_index(t, q, r) * a.wedge_A + a.wedge_j] = v.x;
            }
        }
        __syncthreads(); // the stage is read out before it is refilled
    }
    ldgsts_wait<0>(); // no copy outlives the CTA
}

// ------------------------------------------------------------------------
// Column passes with one lane per tile column (N = 256, 384 and 512).
//
// The tile (N rows x CW columns, dense [N][CW] in shared memory) is
// transformed by 256 threads in two radix stages, N = R1 G (R1 = 16, or 12
// at N = 384; G = 16 at N = 256, else 32):
//   stage 1: thread (column c, residue q < G) holds x[q + G p], p < R1, in
//            registers, applies an R1-point DFT and the twiddle W_N^(q k1),
//            and writes Y[q][k1] back over the R1 elements it read (rows
//            k1 G + q are exactly rows q + G p), so no barrier is needed
//            before the write;
//   stage 2 (after one barrier): thread (c, k1) takes Y[q][k1] over q and
//            applies the G-point DFT: a 16-point DFT in registers (G = 16),
//            or (G = 32) two 16-point DFTs over the even and odd q, held by
//            the two lanes 8 apart, combined by one radix-2 step through a
//            warp shuffle (at N = 384 the last two warps have no k1 < 12 and
//            sit this stage out).
// Lanes of a warp always touch whole 64- or 128-byte row segments of the
// tile, so every shared-memory access is free of bank conflicts, and each
// active thread ends with 16 outputs of its column, at rows tb + ts k (k < 16).
template <int N> __host__ __device__ constexpr bool cols_lanes_ok() { return N == 256 || N == 384 || N == 512; }
// first-stage radix of the lanes passes: 16, or 12 at N = 384 (= 12 x 32)
template <int N> __host__ __device__ constexpr int lanes_r1(int) { return N == 384 ? 12 : 16; }

template <int N, int DIR>
__device__ __forceinline__ bool fft_cols_lanes(float2* __restrict__ buf, const float2* __restrict__ tw,
                                               float2 (&v)[16], int& col, int& tb, int& ts) {
    constexpr int CW = cw_of(N), R1 = lanes_r1<N>(0), G = N / R1;
    static_assert(CW * G == 256, "256 threads: one per (column, residue)");
    const int tid = threadIdx.x;
    {
        const int c = tid % CW, q = tid / CW;
#pragma unroll
        for (int p = 0; p < R1; ++p) v[p] = buf[(q + G * p) * CW + c];
        dft<R1, DIR>(v);
#pragma unroll
        for (int k1 = 1; k1 < R1; ++k1) {
            float2 w = tw[q * k1]; // W_N^(q k1), q k1 < N
            if (DIR > 0) w.y = -w.y;
            v[k1] = cmul(v[k1], w);
        }
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) buf[(k1 * G + q) * CW + c] = v[k1];
    }
    __syncthreads();
    if constexpr (G == 16) {
        const int c = tid % 16, k1 = tid / 16;
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = buf[(k1 * 16 + q) * 16 + c];
        dft16<DIR>(v); // v[k2] = X[k1 + 16 k2]
        col = c;
        tb = k1;
        ts = 16;
        return true;
    } else {
        // q = 2 m + b: E_b = 16-point DFT over m; X[k1 + R1 (k2 + 16 c')] = E_0 + (-1)^c' W_32^k2 E_1
        const int c = tid % 8, b = (tid >> 3) & 1, k1 = tid >> 4;
        const bool active = k1 < R1; // whole warps: k1 = 2 w or 2 w + 1
        if (active) {
#pragma unroll
            for (int m = 0; m < 16; ++m) v[m] = buf[(k1 * 32 + 2 * m + b) * 8 + c];
            dft16<DIR>(v);
        }
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) {
            const float2 f = make_float2(__shfl_xor_sync(0xffffffffu, v[k2].x, 8),
                                         __shfl_xor_sync(0xffffffffu, v[k2].y, 8));
            float2 w = tw[R1 * k2]; // W_N^(R1 k2) = W_32^k2
            if (DIR > 0) w.y = -w.y;
            v[k2] = b == 0 ? cadd(v[k2], cmul(w, f)) : csub(f, cmul(w, v[k2]));
        }
        col = c;
        tb = k1 + 16 * R1 * b;
        ts = R1;
        return active;
    }
}

// The pipelined persistent column pass with fft_cols_lanes: as k_cols_pl
// (tiles copied by 16-byte asynchronous copies into S shared-memory stages,
// S - 1 in flight), with 256 threads and the outputs written straight from
// registers (two or four whole row segments per warp store).  Two tile
// schedules: S = 4 stages, one CTA per SM (133 KB), or S = 3 stages, two CTAs
// per SM (100 KB each), so one CTA's transforms overlap the other's waits.
__host__ __device__ constexpr int cols_lanes_threads() { return 256; }
template <int N, int S> __host__ __device__ constexpr size_t cols_lanes_smem_bytes() {
    return sizeof(float2) * ((size_t)N + (size_t)S * N * cw_of(N));
}
template <int N, int DIR, int OUT, int S>
__global__ void __launch_bounds__(cols_lanes_threads()) k_cols_lanes(ColArgs a, int ntiles) {
    constexpr int NT = cols_lanes_threads();
    constexpr int CW = cw_of(N), M = N / 2;
    constexpr int TILE = N * CW;
    static_assert(cols_lanes_ok<N>(), "N = 256, 384 or 512");
    extern __shared__ float4 smem_raw[];
    float2* tw = reinterpret_cast<float2*>(smem_raw);
    float2* stages = tw + N;
    for (int i = threadIdx.x; i < N; i += NT) tw[i] = a.tw[i];
    auto load = [&](int tile, float2* dst) {
        const ColGeom<N> g(tile + a.tile0, a.axis);
        if (!g.nyq) {
            for (int c = threadIdx.x; c < TILE / 2; c += NT) ldgsts16(dst + 2 * c, a.src + g.at(2 * c));
        } else {
            for (int i = threadIdx.x; i < TILE; i += NT) ldgsts8(dst + i, a.src + g.at(i));
        }
    };
#pragma unroll
    for (int k = 0; k < S - 1; ++k) {
        const int t = blockIdx.x + k * gridDim.x;
        if (t < ntiles) load(t, stages + k * TILE);
        ldgsts_commit();
    }
    for (int k = 0;; ++k) {
        const int tile = blockIdx.x + k * gridDim.x;
        if (tile >= ntiles) break;
        const int nt = blockIdx.x + (k + S - 1) * gridDim.x;
        if (nt < ntiles) load(nt, stages + ((k + S - 1) % S) * TILE);
        ldgsts_commit();
        ldgsts_wait<S - 1>();
        __syncthreads();
        float2* buf = stages + (k % S) * TILE;
        float2 v[16];
        int col, tb, ts;
        const bool active = fft_cols_lanes<N, DIR>(buf, tw, v, col, tb, ts);
        const ColGeom<N> g(tile + a.tile0, a.axis);
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            if (!active) break;
            const int t = tb + ts * kk;
            const int idx = t * CW + col;
            if constexpr (OUT == COL_OUT_PLAIN) {
                a.dst[g.at(idx)] = v[kk];
            } else if constexpr (OUT == COL_OUT_BF16) {
                a.dst_bf16[((long long)(tile + a.tile0) * a.n_ring + a.wslot) * TILE + idx] =
                    __floats2bfloat162_rn(v[kk].x, v[kk].y);
            } else if constexpr (OUT == COL_OUT_RING_F32) {
                a.dst[((long long)(tile + a.tile0) * a.n_ring + a.wslot) * TILE + idx] = v[kk];
            } else {
                const int q = g.nyq ? g.line + col : g.line;
                const int r = g.nyq ? M : g.chunk * CW + col;
                if (t <= q && q <= r) a.wedge_out[wedge_index(t, q, r) * a.wedge_A + a.wedge_j] = v[kk].x;
            }
        }
        __syncthreads(); // the stage is read out before it is refilled
    }
    ldgsts_wait<0>();
}

// ------------------------------------------------------------------------
// Column passes with the tiles moved by tensor-map TMA (N = 256 and 512):
// the transform is fft_cols_lanes; a full tile is one box (two from N = 384:
// a box holds at most 256 rows) of the half spectrum seen as a 3D tensor
// [p][q][2 NRP floats], copied by cp.async.bulk.tensor into one of S
// shared-memory stages, completion counted on the stage's mbarrier, issued
// by one thread S - 1 tiles ahead.  Nyquist tiles (CW single columns of CW
// lines, not a box of contiguous columns) are loaded by the threads
// themselves when their turn comes.  Every wait is bounded: a wait that
// gives up sets bit 8 of the error word; the CTA then waits once more (also
// bounded) for each copy it has in flight and returns.
template <int N, int S> __host__ __device__ constexpr size_t cols_tma_smem_bytes() {
    return (size_t)S * N * cw_of(N) * sizeof(float2) + (size_t)N * sizeof(float2) + (size_t)S * 8 + 128;
}
template <int N, int DIR, int OUT, int S>
__global__ void __launch_bounds__(cols_lanes_threads()) k_cols_tma(ColArgs a, int ntiles,
                                                                    const __grid_constant__ CUtensorMap tmap) {
    constexpr int NT = cols_lanes_threads();
    constexpr int CW = cw_of(N), M = N / 2, TILE = N * CW, NCH = M / CW;
    constexpr int BOX = N > 256 ? N / 2 : N, NBOX = N / BOX; // a box holds at most 256 rows
    static_assert(BOX <= 256 && N % BOX == 0, "whole boxes of at most 256 rows");
    constexpr unsigned TILE_BYTES = TILE * sizeof(float2);
    static_assert(cols_lanes_ok<N>(), "N = 256, 384 or 512");
    extern __shared__ unsigned char smem_tma[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_tma) + 127) & ~uintptr_t(127));
    float2* stages = reinterpret_cast<float2*>(sm); // S tiles, each 128-byte aligned
    float2* tw = stages + S * TILE;
    unsigned long long* full = reinterpret_cast<unsigned long long*>(tw + N);
    __shared__ int s_fail;
    if (threadIdx.x == 0) {
        s_fail = 0;
        for (int k = 0; k < S; ++k) mbar_init(smem_u32(&full[k]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = threadIdx.x; i < N; i += NT) tw[i] = a.tw[i];
    __syncthreads();
    auto is_nyq = [&](int tile) { return tile + a.tile0 >= N * NCH; };
    auto issue = [&](int tile, int st) { // thread 0; full tiles only
        const int t = tile + a.tile0, line = t / NCH, chunk = t % NCH;
        const unsigned bar = smem_u32(&full[st]);
        mbar_expect_tx(bar, TILE_BYTES);
#pragma unroll
        for (int b = 0; b < NBOX; ++b) {
            const unsigned dst = smem_u32(stages + st * TILE + b * BOX * CW);
            // coordinates (float along r, q, p): y pass (axis 0) p = line, x pass q = line
            if (a.axis == 0) tma_load_3d(dst, &tmap, 2 * chunk * CW, b * BOX, line, bar);
            else tma_load_3d(dst, &tmap, 2 * chunk * CW, line, b * BOX, bar);
        }
    };
    if (threadIdx.x == 0) {
        for (int k = 0; k < S - 1; ++k) {
            const int t = blockIdx.x + k * gridDim.x;
            if (t < ntiles && !is_nyq(t)) issue(t, k);
        }
    }
    unsigned phase = 0; // bit st: parity of the next completion of stage st
    for (int k = 0;; ++k) {
        const int tile = blockIdx.x + k * gridDim.x;
        if (tile >= ntiles) break;
        const int st = k % S;
        // refill the stage of tile k - 1 (every thread is done with it: the
        // barrier that ended tile k - 1)
        if (threadIdx.x == 0) {
            const int nt = blockIdx.x + (k + S - 1) * gridDim.x;
            if (nt < ntiles && !is_nyq(nt)) {
                fence_proxy_async();
                issue(nt, (k + S - 1) % S);
            }
        }
        float2* buf = stages + st * TILE;
        const ColGeom<N> g(tile + a.tile0, a.axis);
        bool ok = true;
        if (g.nyq) {
            for (int i = threadIdx.x; i < TILE; i += NT) buf[i] = a.src[g.at(i)];
            __syncthreads();
        } else {
            ok = mbar_wait_bounded(smem_u32(&full[st]), (phase >> st) & 1u);
            phase ^= 1u << st;
        }
        if (__syncthreads_or(!ok)) {
            // give every copy still in flight (this tile's, and those issued
            // ahead) a second bounded wait before the shared memory goes away
            if (threadIdx.x == 0) {
                if (!g.nyq) mbar_wait_bounded(smem_u32(&full[st]), ((phase >> st) & 1u) ^ 1u);
                for (int d = 1; d < S; ++d) {
                    const int t2 = blockIdx.x + (k + d) * gridDim.x;
                    const int s2 = (k + d) % S;
                    if (t2 < ntiles && !is_nyq(t2)) mbar_wait_bounded(smem_u32(&full[s2]), (phase >> s2) & 1u);
                }
                if (a.err) atomicOr(a.err, 8);
            }
            return;
        }
        float2 v[16];
        int col, tb, ts;
        const bool active = fft_cols_lanes<N, DIR>(buf, tw, v, col, tb, ts);
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            if (!active) break;
            const int t = tb + ts * kk;
            const int idx = t * CW + col;
            if constexpr (OUT == COL_OUT_PLAIN) {
                a.dst[g.at(idx)] = v[kk];
            } else if constexpr (OUT == COL_OUT_BF16) {
                a.dst_bf16[((long long)(tile + a.tile0) * a.n_ring + a.wslot) * TILE + idx] =
                    __floats2bfloat162_rn(v[kk].x, v[kk].y);
            } else if constexpr (OUT == COL_OUT_RING_F32) {
                a.dst[((long long)(tile + a.tile0) * a.n_ring + a.wslot) * TILE + idx] = v[kk];
            } else {
                const int q = g.nyq ? g.line + col : g.line;
                const int r = g.nyq ? M : g.chunk * CW + col;
                if (t <= q && q <= r) a.wedge_out[wedge_index(t, q, r) * a.wedge_A + a.wedge_j] = v[kk].x;
            }
        }
        __syncthreads(); // the stage is read out before it is refilled
    }
}

// ------------------------------------------------------------------------
// z passes with one row pair per group of G lanes (N = 256: a half warp,
// N = 384 and 512: a warp).  The two real rows a, b of a pair are
// transformed as one complex row z = a + i b (Eq. 12 along z), N = R1 G:
//   stage 1: lane q holds z[q + G p], p < R1: R1-point DFT, twiddle
//            W_N^(q k1), written to a warp-private exchange buffer at
//            k1 (G + 1) + q (the skew keeps both directions free of bank
//            conflicts);
//   stage 2: G = 16: lane k1 reads Y[q][k1] over q, 16-point DFT:
//            Z[k1 + 16 k2]; G = 32: lane (k1, b) reads the even (b = 0) or
//            odd q, 16-point DFT, and one radix-2 step with lane ^ 1 through
//            a shuffle: Z[k1 + R1 k2 + 16 R1 b] (at N = 384 lanes 24..31
//            have no k1 < 12 and sit this stage out).
// Only warp-level synchronisation is needed: a group never waits for the
// rest of the block.  Row pairs are assigned per warp, so both half warps of
// a warp run the same number of iterations.
template <int N> __host__ __device__ constexpr bool rows_lanes_ok() { return N == 256 || N == 384 || N == 512; }
constexpr int kRowsLanesThreads = 256;
template <int N> __host__ __device__ constexpr int rows_lanes_g() { return N / lanes_r1<N>(0); }
template <int N> __host__ __device__ constexpr int rows_lanes_ex() {
    // float2 per group's exchange buffer: the skewed R1 x G exchange, or Z
    // in natural order plus two, or both half spectra
    return lanes_r1<N>(0) * (rows_lanes_g<N>() + 1) > N + 2 ? lanes_r1<N>(0) * (rows_lanes_g<N>() + 1) : N + 2;
}
template <int N> __host__ __device__ constexpr size_t rows_lanes_smem_bytes() {
    return sizeof(float2) * ((size_t)N + (size_t)(kRowsLanesThreads / rows_lanes_g<N>()) * rows_lanes_ex<N>());
}

// In: v[p] = z[q + G p] of this lane (q = lane within its group).  Out: this
// lane's 16 outputs Z[t0 + ts k], k < 16 (t0, ts returned; active false:
// the lane holds no outputs).
template <int N, int DIR>
__device__ __forceinline__ bool fft_row_lanes(float2 (&v)[16], float2* __restrict__ ex, const float2* __restrict__ tw,
                                              int q, int& t0, int& ts) {
    constexpr int R1 = lanes_r1<N>(0), G = N / R1, XS = G + 1;
    dft<R1, DIR>(v);
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) {
        float2 w = tw[q * k1];
        if (DIR > 0) w.y = -w.y;
        v[k1] = cmul(v[k1], w);
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) ex[k1 * XS + q] = v[k1];
    __syncwarp();
    if constexpr (G == 16) {
#pragma unroll
        for (int qq = 0; qq < 16; ++qq) v[qq] = ex[q * XS + qq];
        dft16<DIR>(v);
        __syncwarp();
        t0 = q;
        ts = 16;
        return true;
    } else {
        const int k1 = q >> 1, b = q & 1;
        const bool active = k1 < R1;
        if (active) {
#pragma unroll
            for (int m = 0; m < 16; ++m) v[m] = ex[k1 * XS + 2 * m + b];
            dft16<DIR>(v);
        }
#pragma unroll
        for (int k2 = 0; k2 < 16; ++k2) {
            const float2 f = make_float2(__shfl_xor_sync(0xffffffffu, v[k2].x, 1),
                                         __shfl_xor_sync(0xffffffffu, v[k2].y, 1));
            float2 w = tw[R1 * k2]; // W_N^(R1 k2) = W_32^k2
            if (DIR > 0) w.y = -w.y;
            v[k2] = b == 0 ? cadd(v[k2], cmul(w, f)) : csub(f, cmul(w, v[k2]));
        }
        __syncwarp();
        t0 = k1 + 16 * R1 * b;
        ts = R1;
        return active;
    }
}

// z forward, real -> complex: int64 deposit grid (times the slot's scale,
// cleared after reading when zero_in) or float input; output rows of NRP.
template <int N, int IN>
__global__ void __launch_bounds__(kRowsLanesThreads, 2) k_rows_r2c_lanes(RowR2CArgs a, long long npairs) {
    constexpr int R1 = lanes_r1<N>(0), G = N / R1, PW = 32 / G, NRP = nrp_of(N), H = N / 2 + 1, EX = rows_lanes_ex<N>();
    static_assert(IN == ROW_IN_I64 || IN == ROW_IN_F32, "grid or float input");
    extern __shared__ float4 smem_raw[];
    float2* tw = reinterpret_cast<float2*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane / G, q = lane % G;
    float2* ex = tw + N + (warp * PW + grp) * EX;
    for (int i = threadIdx.x; i < N; i += kRowsLanesThreads) tw[i] = a.tw[i];
    float scale = 1.0f;
    unsigned cur = 0;
    if constexpr (IN == ROW_IN_I64) {
        const double Su = a.slot_S[a.slot];
        const long long tot = a.slot_total[a.slot];
        // as k_rows_r2c: S per unit (FP32 history), 1 / total (BF16 history)
        scale = a.bf16 ? (tot > 0 ? (float)(1.0 / (double)tot) : 0.0f) : (float)Su;
        if (a.rowstamp) cur = *a.stamp;
    }
    const long long nwarps = (long long)gridDim.x * (kRowsLanesThreads / 32);
    long long u = (long long)blockIdx.x * (kRowsLanesThreads / 32) + warp;
    // the row stamps of a warp's rows, loaded one iteration ahead (lane l < 2 PW: row 2 u PW + l)
    unsigned stamp_next = 0;
    if constexpr (IN == ROW_IN_I64)
        if (a.rowstamp && lane < 2 * PW && u * PW < npairs) stamp_next = a.rowstamp[2 * u * PW + lane];
    __syncthreads();
    for (; u * PW < npairs; u += nwarps) {
        const long long rp = u * PW + grp; // npairs is a multiple of PW: every group of the warp has a pair
        const long long ra = 2 * rp * N, rb = ra + N;
        float2 v[16];
        if constexpr (IN == ROW_IN_I64) {
            if (a.rowstamp) {
                // the warp's 2 PW rows (2 u PW ... 2 u PW + 2 PW - 1 < 2 npairs);
                // none with a share of this push: zero half spectra, no loads
                const bool mine = lane < 2 * PW && stamp_next == cur;
                const long long un = u + nwarps;
                stamp_next = (lane < 2 * PW && un * PW < npairs) ? a.rowstamp[2 * un * PW + lane] : 0u;
                if (!__any_sync(0xffffffffu, mine)) {
                    float2* da = a.dst + (2 * rp) * NRP;
                    float2* db = da + NRP;
#pragma unroll
                    for (int m = 0; m < (H + G - 1) / G; ++m) {
                        const int k = q + G * m;
                        if (k < H) {
                            da[k] = make_float2(0.f, 0.f);
                            db[k] = make_float2(0.f, 0.f);
                        }
                    }
                    continue;
                }
            }
            long long xa[R1], xb[R1];
#pragma unroll
            for (int p = 0; p < R1; ++p) {
                xa[p] = a.grid[ra + q + G * p];
                xb[p] = a.grid[rb + q + G * p];
            }
            if (a.zero_in) {
                long long* g = const_cast<long long*>(a.grid);
#pragma unroll
                for (int p = 0; p < R1; ++p) {
                    g[ra + q + G * p] = 0;
                    g[rb + q + G * p] = 0;
                }
            }
#pragma unroll
            for (int p = 0; p < R1; ++p) v[p] = make_float2(__ll2float_rn(xa[p]) * scale, __ll2float_rn(xb[p]) * scale);
        } else {
#pragma unroll
            for (int p = 0; p < R1; ++p) v[p] = make_float2(a.fin[ra + q + G * p], a.fin[rb + q + G * p]);
        }
        int t0, ts;
        const bool active = fft_row_lanes<N, -1>(v, ex, tw, q, t0, ts);
        // Z in natural order, then the two real rows' half spectra:
        // X_a = (Z_k + conj Z_{N-k}) / 2, X_b = (Z_k - conj Z_{N-k}) / (2 i)
        if (active) {
#pragma unroll
            for (int k = 0; k < 16; ++k) ex[t0 + ts * k] = v[k];
        }
        __syncwarp();
        float2* da = a.dst + (2 * rp) * NRP;
        float2* db = da + NRP;
#pragma unroll
        for (int m = 0; m < (H + G - 1) / G; ++m) {
            const int k = q + G * m;
            if (k < H) {
                const float2 zk = ex[k], zn = ex[k == 0 ? 0 : N - k];
                da[k] = make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
                db[k] = make_float2(0.5f * (zk.y + zn.y), 0.5f * (zn.x - zk.x));
            }
        }
        __syncwarp(); // the exchange buffer is free for the next pair
    }
}

// z inverse, complex -> real, times `scale`: rows of NRP in, N floats out.
template <int N>
__global__ void __launch_bounds__(kRowsLanesThreads, 2) k_rows_c2r_lanes(RowC2RArgs a, long long npairs) {
    constexpr int R1 = lanes_r1<N>(0), G = N / R1, PW = 32 / G, NRP = nrp_of(N), H = N / 2 + 1, EX = rows_lanes_ex<N>();
    static_assert(2 * H <= EX, "both half spectra fit the exchange buffer");
    extern __shared__ float4 smem_raw[];
    float2* tw = reinterpret_cast<float2*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane / G, q = lane % G;
    float2* ex = tw + N + (warp * PW + grp) * EX;
    for (int i = threadIdx.x; i < N; i += kRowsLanesThreads) tw[i] = a.tw[i];
    __syncthreads();
    const long long nwarps = (long long)gridDim.x * (kRowsLanesThreads / 32);
    for (long long u = (long long)blockIdx.x * (kRowsLanesThreads / 32) + warp; u * PW < npairs; u += nwarps) {
        const long long rp = u * PW + grp;
        const float2* sa = a.src + (2 * rp) * NRP;
        const float2* sb = sa + NRP;
        float2* xa = ex;
        float2* xb = ex + H;
#pragma unroll
        for (int m = 0; m < (H + G - 1) / G; ++m) {
            const int k = q + G * m;
            if (k < H) {
                float2 A = sa[k], B = sb[k];
                if (k == 0 || k == N / 2) {
                    A.y = 0.f;
                    B.y = 0.f;
                }
                xa[k] = A;
                xb[k] = B;
            }
        }
        __syncwarp();
        // Z_n = X_a(n) + i X_b(n), with the Hermitian extension X(N - k) = conj X(k)
        float2 v[16];
#pragma unroll
        for (int p = 0; p < R1; ++p) {
            const int n = q + G * p;
            if (n < H) {
                const float2 A = xa[n], B = xb[n];
                v[p] = make_float2(A.x - B.y, A.y + B.x);
            } else {
                const float2 A = xa[N - n], B = xb[N - n];
                v[p] = make_float2(A.x + B.y, B.x - A.y);
            }
        }
        __syncwarp();
        int t0, ts;
        const bool active = fft_row_lanes<N, 1>(v, ex, tw, q, t0, ts);
        float* oa = a.out + (2 * rp) * N;
        float* ob = oa + N;
        if (active) {
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                oa[t0 + ts * k] = v[k].x * a.scale;
                ob[t0 + ts * k] = v[k].y * a.scale;
            }
        }
    }
}

// ------------------------------------------------------------------------
// z rows, complex -> real, persistent with the next block's loads in flight.
template <int N>
__global__ void __launch_bounds__(kThreads) k_rows_c2r(RowC2RArgs a, int nblocks) {
    constexpr int B = row_pairs_of(N), BP = odd_pad(B), NRP = nrp_of(N), H = N / 2 + 1;
    constexpr int TILE = B * H, PER = (TILE + kThreads - 1) / kThreads;
    extern __shared__ float4 smem_raw[];
    float2* tw = reinterpret_cast<float2*>(smem_raw);
    float2* buf = tw + N;
    auto fetch = [&](int blk, float2* xa, float2* xb) {
        const long long row0 = (long long)blk * (2 * B);
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int idx = threadIdx.x + i * kThreads;
            const int pair = idx / H, k = idx % H;
            const long long ra = row0 + 2 * pair, rb = ra + 1;
            const bool ok = TILE % kThreads == 0 || idx < TILE;
            xa[i] = (ok && ra < a.nrows) ? a.src[ra * NRP + k] : make_float2(0.f, 0.f);
            xb[i] = (ok && rb < a.nrows) ? a.src[rb * NRP + k] : make_float2(0.f, 0.f);
        }
    };
    for (int i = threadIdx.x; i < N; i += kThreads) tw[i] = a.tw[i];
    float2 ca[PER], cb[PER], na[PER], nb[PER];
    int blk = blockIdx.x;
    if (blk < nblocks) fetch(blk, ca, cb);
    while (blk < nblocks) {
        const int next = blk + gridDim.x;
        if (next < nblocks) fetch(next, na, nb);
        __syncthreads();
        // Z_k = X_a(k) + i X_b(k), with the Hermitian extension X(N-k) = conj X(k)
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int idx = threadIdx.x + i * kThreads;
            if (!(TILE % kThreads == 0 || idx < TILE)) continue;
            const int pair = idx / H, k = idx % H;
            float2 A = ca[i], Bv = cb[i];
            if (k == 0 || k == N / 2) { A.y = 0.f; Bv.y = 0.f; }
            buf[k * BP + pair] = make_float2(A.x - Bv.y, A.y + Bv.x);
            if (k > 0 && k < N / 2) buf[(N - k) * BP + pair] = make_float2(A.x + Bv.y, Bv.x - A.y);
        }
        __syncthreads();
        fft_smem<N, 1, B, BP>(buf, tw);
        const long long row0 = (long long)blk * (2 * B);
        for (int idx = threadIdx.x; idx < 2 * B * N; idx += kThreads) {
            const int rr = idx / N, t = idx % N;
            const long long grow = row0 + rr;
            if (grow >= a.nrows) continue;
            const float2 v = buf[t * BP + (rr >> 1)];
            a.out[grow * N + t] = ((rr & 1) ? v.y : v.x) * a.scale;
        }
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            ca[i] = na[i];
            cb[i] = nb[i];
        }
        blk = next;
    }
}

// ------------------------------------------------------------------------
// Pipelined z passes (N >= 256, where N^2 rows split into whole blocks of B
// row pairs): the rows of a block are one contiguous run in memory, copied by
// 16-byte asynchronous copies into one of S shared-memory stages, S - 1 blocks
// in flight while one is packed into the transform buffer and transformed.
// Forward: int64 deposit grid or float input (the Green's-function wedge
// gather stays with k_rows_r2c); inverse: half-spectrum rows of NRP.
__host__ __device__ constexpr int rows_pl_stages(int n) { return 4; }
template <int N, int E> __host__ __device__ constexpr size_t rows_pl_stage_bytes() {
    return (size_t)2 * row_pairs_of(N) * N * E;
}
template <int N, int IN> __host__ __device__ constexpr size_t rows_r2c_pl_smem_bytes() {
    return sizeof(float2) * ((size_t)N + (size_t)N * odd_pad(row_pairs_of(N))) +
           (size_t)rows_pl_stages(N) * rows_pl_stage_bytes<N, IN == ROW_IN_I64 ? 8 : 4>();
}
template <int N> __host__ __device__ constexpr size_t rows_c2r_pl_smem_bytes() {
    return sizeof(float2) * ((size_t)N + (size_t)N * odd_pad(row_pairs_of(N))) +
           (size_t)rows_pl_stages(N) * 2 * row_pairs_of(N) * nrp_of(N) * sizeof(float2);
}

template <int N, int IN>
__global__ void __launch_bounds__(kThreads) k_rows_r2c_pl(RowR2CArgs a, int nblocks) {
    constexpr int B = row_pairs_of(N), BP = odd_pad(B), NRP = nrp_of(N), H = N / 2 + 1, S = rows_pl_stages(N);
    constexpr int E = IN == ROW_IN_I64 ? 8 : 4, R2 = 2 * B;
    constexpr int SB = (int)rows_pl_stage_bytes<N, E>(), CH = SB / 16;
    static_assert(IN != ROW_IN_WEDGE && (N * N) % R2 == 0 && SB % 16 == 0, "whole contiguous blocks");
    extern __shared__ float4 smem_raw[];
    float2* tw = reinterpret_cast<float2*>(smem_raw);
    float2* buf = tw + N;
    unsigned char* stages = reinterpret_cast<unsigned char*>(buf + N * BP); // 16-byte aligned
    float scale = 1.0f;
    if constexpr (IN == ROW_IN_I64) {
        // as k_rows_r2c: S per unit (FP32 history), 1 / total (BF16 history)
        const double Su = a.slot_S[a.slot];
        const long long tot = a.slot_total[a.slot];
        scale = a.bf16 ? (tot > 0 ? (float)(1.0 / (double)tot) : 0.0f) : (float)Su;
    }
    const unsigned char* src = IN == ROW_IN_I64 ? reinterpret_cast<const unsigned char*>(a.grid)
                                                : reinterpret_cast<const unsigned char*>(a.fin);
    auto load = [&](int blk, unsigned char* dst) {
        const unsigned char* s = src + (size_t)blk * SB;
        for (int c = threadIdx.x; c < CH; c += kThreads) ldgsts16(dst + 16 * c, s + 16 * c);
    };
    for (int i = threadIdx.x; i < N; i += kThreads) tw[i] = a.tw[i];
#pragma unroll
    for (int k = 0; k < S - 1; ++k) {
        const int b = blockIdx.x + k * gridDim.x;
        if (b < nblocks) load(b, stages + k * SB);
        ldgsts_commit();
    }
    float* bf = reinterpret_cast<float*>(buf);
    for (int k = 0;; ++k) {
        const int blk = blockIdx.x + k * gridDim.x;
        if (blk >= nblocks) break;
        const int nb = blockIdx.x + (k + S - 1) * gridDim.x;
        if (nb < nblocks) load(nb, stages + ((k + S - 1) % S) * SB);
        ldgsts_commit();
        ldgsts_wait<S - 1>();
        __syncthreads(); // block k has landed; the previous block has left buf
        const unsigned char* st = stages + (k % S) * SB;
        if constexpr (IN == ROW_IN_I64) {
            // the block's grid cells are read: zero them for the next deposit
            if (a.zero_in) {
                int4* g = reinterpret_cast<int4*>(const_cast<long long*>(a.grid)) + (size_t)blk * CH;
                for (int c = threadIdx.x; c < CH; c += kThreads) g[c] = make_int4(0, 0, 0, 0);
            }
        }
        for (int idx = threadIdx.x; idx < R2 * N; idx += kThreads) {
            const int rr = idx / N, t = idx % N;
            float v;
            if constexpr (IN == ROW_IN_I64) v = __ll2float_rn(reinterpret_cast<const long long*>(st)[idx]) * scale;
            else v = reinterpret_cast<const float*>(st)[idx];
            bf[2 * (t * BP + (rr >> 1)) + (rr & 1)] = v; // row pair rr/2, real / imaginary part
        }
        __syncthreads();
        fft_smem<N, -1, B, BP>(buf, tw);
        const long long row0 = (long long)blk * R2;
        for (int idx = threadIdx.x; idx < R2 * H; idx += kThreads) {
            const int rr = idx / H, kk = idx % H;
            const int pair = rr >> 1;
            const float2 zk = buf[kk * BP + pair];
            const float2 zn = buf[(kk == 0 ? 0 : N - kk) * BP + pair];
            float2 x;
            if ((rr & 1) == 0) x = make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
            else x = make_float2(0.5f * (zk.y + zn.y), 0.5f * (zn.x - zk.x));
            a.dst[(row0 + rr) * NRP + kk] = x;
        }
        __syncthreads(); // buf and the stage are free again
    }
    ldgsts_wait<0>();
}

template <int N>
__global__ void __launch_bounds__(kThreads) k_rows_c2r_pl(RowC2RArgs a, int nblocks) {
    constexpr int B = row_pairs_of(N), BP = odd_pad(B), NRP = nrp_of(N), H = N / 2 + 1, S = rows_pl_stages(N);
    constexpr int R2 = 2 * B, SE = R2 * NRP, CH = SE / 2; // stage elements, 16-byte chunks
    static_assert((N * N) % R2 == 0 && NRP % 2 == 0, "whole contiguous blocks");
    extern __shared__ float4 smem_raw[];
    float2* tw = reinterpret_cast<float2*>(smem_raw);
    float2* buf = tw + N;
    float2* stages = buf + N * BP;
    auto load = [&](int blk, float2* dst) {
        const float2* s = a.src + (size_t)blk * SE;
        for (int c = threadIdx.x; c < CH; c += kThreads) ldgsts16(dst + 2 * c, s + 2 * c);
    };
    for (int i = threadIdx.x; i < N; i += kThreads) tw[i] = a.tw[i];
#pragma unroll
    for (int k = 0; k < S - 1; ++k) {
        const int b = blockIdx.x + k * gridDim.x;
        if (b < nblocks) load(b, stages + k * SE);
        ldgsts_commit();
    }
    for (int k = 0;; ++k) {
        const int blk = blockIdx.x + k * gridDim.x;
        if (blk >= nblocks) break;
        const int nb = blockIdx.x + (k + S - 1) * gridDim.x;
        if (nb < nblocks) load(nb, stages + ((k + S - 1) % S) * SE);
        ldgsts_commit();
        ldgsts_wait<S - 1>();
        __syncthreads();
        const float2* st = stages + (k % S) * SE;
        // Z_k = X_a(k) + i X_b(k), with the Hermitian extension X(N-k) = conj X(k)
        for (int idx = threadIdx.x; idx < B * H; idx += kThreads) {
            const int pair = idx / H, kk = idx % H;
            float2 A = st[(2 * pair) * NRP + kk], Bv = st[(2 * pair + 1) * NRP + kk];
            if (kk == 0 || kk == N / 2) { A.y = 0.f; Bv.y = 0.f; }
            buf[kk * BP + pair] = make_float2(A.x - Bv.y, A.y + Bv.x);
            if (kk > 0 && kk < N / 2) buf[(N - kk) * BP + pair] = make_float2(A.x + Bv.y, Bv.x - A.y);
        }
        __syncthreads();
        fft_smem<N, 1, B, BP>(buf, tw);
        const long long row0 = (long long)blk * R2;
        for (int idx = threadIdx.x; idx < R2 * N; idx += kThreads) {
            const int rr = idx / N, t = idx % N;
            const float2 v = buf[t * BP + (rr >> 1)];
            a.out[(row0 + rr) * N + t] = ((rr & 1) ? v.y : v.x) * a.scale;
        }
        __syncthreads();
    }
    ldgsts_wait<0>();
}

// ------------------------------------------------------------------------
// Plane kernels (grids whose half plane fits in shared memory, N <= 192):
// one CTA per x-plane does the z and y axes of the forward (or inverse)
// transform in shared memory, replacing two full passes through memory.
// Layout: plane[y * H + k], H = N/2 + 1 (odd, so both axes are bank-conflict
// free); the z transform runs on row pairs in the same buffer as [t * H + pair].
__host__ __device__ constexpr int plane_threads_of(int n) { return n == 128 ? 1024 : (n >= 64 ? 512 : 256); }
template <int N> __host__ __device__ constexpr size_t plane_smem_bytes() {
    return sizeof(float2) * (N + (size_t)N * (N / 2 + 1));
}
template <int N> __host__ __device__ constexpr bool plane_ok() { return N <= 192 && plane_smem_bytes<N>() <= 227 * 1024; }

template <int N, int IN>
__global__ void __launch_bounds__(plane_threads_of(N)) k_plane_r2c(RowR2CArgs a) {
    constexpr int NT = plane_threads_of(N), H = N / 2 + 1, NRP = nrp_of(N), P = N / 2;
    constexpr int TILE = N * N, PER = (TILE + NT - 1) / NT;
    constexpr int UN = P * H, UPER = (UN + NT - 1) / NT;
    extern __shared__ float4 smem_raw[];
    float2* tw = reinterpret_cast<float2*>(smem_raw);
    float2* pl = tw + N;
    const int x = blockIdx.x;
    float scale = 1.0f;
    double gsc = 1.0;
    if constexpr (IN == ROW_IN_I64) {
        const double S = a.slot_S[a.slot];
        const long long tot = a.slot_total[a.slot];
        scale = a.bf16 ? (tot > 0 ? (float)(1.0 / (double)tot) : 0.0f) : (float)S;
    }
    if constexpr (IN == ROW_IN_WEDGE) gsc = *a.gscale;
    float val[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int idx = threadIdx.x + i * NT;
        val[i] = 0.0f;
        if (TILE % NT == 0 || idx < TILE) {
            const int y = idx / N, t = idx % N;
            const long long g = ((long long)x * N + y) * N + t;
            if constexpr (IN == ROW_IN_I64) val[i] = __ll2float_rn(a.grid[g]) * scale;
            else if constexpr (IN == ROW_IN_F32) val[i] = a.fin[g];
            else {
                const int fx = x <= N - x ? x : N - x, fy = y <= N - y ? y : N - y, fz = t <= N - t ? t : N - t;
                const int mx = fx > fy ? (fx > fz ? fx : fz) : (fy > fz ? fy : fz);
                val[i] = mx <= a.near_r ? 0.0f : (float)(a.gw[wedge_of(x, y, t, N)] * gsc);
            }
        }
    }
    for (int i = threadIdx.x; i < N; i += NT) tw[i] = a.tw[i];
    float* pf = reinterpret_cast<float*>(pl);
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int idx = threadIdx.x + i * NT;
        if (TILE % NT == 0 || idx < TILE) {
            const int y = idx / N, t = idx % N;
            pf[2 * (t * H + (y >> 1)) + (y & 1)] = val[i]; // row pair y/2, real / imaginary part
        }
    }
    __syncthreads();
    fft_smem<N, -1, P, H, NT>(pl, tw); // z: N/2 complex row pairs
    // unpack pairs into the half plane [y][k]
    float2 xa[UPER], xb[UPER];
#pragma unroll
    for (int i = 0; i < UPER; ++i) {
        const int idx = threadIdx.x + i * NT;
        if (UN % NT == 0 || idx < UN) {
            const int pair = idx / H, k = idx % H;
            const float2 zk = pl[k * H + pair];
            const float2 zn = pl[(k == 0 ? 0 : N - k) * H + pair];
            xa[i] = make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
            xb[i] = make_float2(0.5f * (zk.y + zn.y), 0.5f * (zn.x - zk.x));
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < UPER; ++i) {
        const int idx = threadIdx.x + i * NT;
        if (UN % NT == 0 || idx < UN) {
            const int pair = idx / H, k = idx % H;
            pl[(2 * pair) * H + k] = xa[i];
            pl[(2 * pair + 1) * H + k] = xb[i];
        }
    }
    __syncthreads();
    fft_smem<N, -1, H, H, NT>(pl, tw); // y: the H columns of the half plane
    for (int idx = threadIdx.x; idx < N * H; idx += NT) {
        const int y = idx / H, k = idx % H;
        a.dst[((long long)x * N + y) * NRP + k] = pl[y * H + k];
    }
}

template <int N>
__global__ void __launch_bounds__(plane_threads_of(N)) k_plane_c2r(RowC2RArgs a) {
    constexpr int NT = plane_threads_of(N), H = N / 2 + 1, NRP = nrp_of(N), P = N / 2;
    constexpr int LD = N * H, LPER = (LD + NT - 1) / NT;
    constexpr int UN = P * H, UPER = (UN + NT - 1) / NT;
    if (blockIdx.x >= N) {
        plane_near_ctas<N, NT>(a.near);
        return;
    }
    extern __shared__ float4 smem_raw[];
    float2* tw = reinterpret_cast<float2*>(smem_raw);
    float2* pl = tw + N;
    const int x = blockIdx.x;
    float2 v[LPER];
#pragma unroll
    for (int i = 0; i < LPER; ++i) {
        const int idx = threadIdx.x + i * NT;
        if (LD % NT == 0 || idx < LD) {
            const int y = idx / H, k = idx % H;
            v[i] = a.src[((long long)x * N + y) * NRP + k];
        }
    }
    for (int i = threadIdx.x; i < N; i += NT) tw[i] = a.tw[i];
#pragma unroll
    for (int i = 0; i < LPER; ++i) {
        const int idx = threadIdx.x + i * NT;
        if (LD % NT == 0 || idx < LD) pl[idx] = v[i]; // [y][k]
    }
    __syncthreads();
    fft_smem<N, 1, H, H, NT>(pl, tw); // y inverse
    // pack rows (2 pair, 2 pair + 1) into Z_k = X_a(k) + i X_b(k), Hermitian-extended in k
    float2 z0[UPER], z1[UPER];
#pragma unroll
    for (int i = 0; i < UPER; ++i) {
        const int idx = threadIdx.x + i * NT;
        if (UN % NT == 0 || idx < UN) {
            const int pair = idx / H, k = idx % H;
            float2 A = pl[(2 * pair) * H + k], B = pl[(2 * pair + 1) * H + k];
            if (k == 0 || k == N / 2) { A.y = 0.f; B.y = 0.f; }
            z0[i] = make_float2(A.x - B.y, A.y + B.x);
            z1[i] = make_float2(A.x + B.y, B.x - A.y);
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < UPER; ++i) {
        const int idx = threadIdx.x + i * NT;
        if (UN % NT == 0 || idx < UN) {
            const int pair = idx / H, k = idx % H;
            pl[k * H + pair] = z0[i];
            if (k > 0 && k < N / 2) pl[(N - k) * H + pair] = z1[i];
        }
    }
    __syncthreads();
    fft_smem<N, 1, P, H, NT>(pl, tw); // z inverse on row pairs
    for (int idx = threadIdx.x; idx < N * N; idx += NT) {
        const int y = idx / N, t = idx % N;
        const float2 w = pl[t * H + (y >> 1)];
        a.out[((long long)x * N + y) * N + t] = ((y & 1) ? w.y : w.x) * a.scale;
    }
}

// ------------------------------------------------------------------------
// Plane kernels with the transforms in registers (N = R1 G: R1 = 16, or 12
// at N = 96 and 192).  A length-N transform is an R1-point DFT per residue
// q < G over x[q + G p], the twiddle W_N^(q k1), and a G-point DFT per k1
// over q, giving X[k1 + R1 k2].  Forward, z: a group of G lanes takes one
// pair of z rows straight from global memory (lane q holds z[q + G p]),
// exchanges once between the two stages through the pair's own two rows of
// the plane buffer, unpacks the two real rows' half spectra there and
// writes them as rows 2u, 2u + 1 of the plane [y][k] (row stride PS).  y:
// item (column c, residue q) runs the first stage in place on rows q + G p;
// after one barrier item (c, k1) runs the second and writes Y[k1 + R1 k2]
// straight to global memory.  This moves about a third of the shared-memory
// bytes of the staged plane kernels (no staging of the input, no
// Stockham stage round trips).
// Item `it` of a y stage over the H = N/2 + 1 columns and `rows` rows: the
// N/2 regular columns first, row by row (whole warps per row from N = 64,
// so a warp's accesses stay in one row), then the Nyquist column (c = N/2).
template <int N>
__device__ __forceinline__ void plane_item(int it, int rows, int& c, int& r) {
    constexpr int M = N / 2;
    if (it < M * rows) {
        c = it % M;
        r = it / M;
    } else {
        c = M;
        r = it - M * rows;
    }
}

template <int N> __host__ __device__ constexpr bool plane_lanes_ok() {
    return N == 32 || N == 64 || N == 96 || N == 128 || N == 192;
}
template <int N> __host__ __device__ constexpr int plane_lanes_r1() { return (N == 96 || N == 192) ? 12 : 16; }
template <int N> __host__ __device__ constexpr int plane_lanes_threads() {
    return N == 32 ? 288 : (N == 64 || N == 128) ? 544 : 608;
}
// Row stride (float2): at least H, room for a pair's exchange in two rows
// (R1 (G + 1) skewed, or Z in natural order, N + 2), and 4 mod 8, so that
// the unpack stores of a warp's lane groups (rows 2 PS apart) fall on
// distinct bank pairs.
template <int N> __host__ __device__ constexpr int plane_lanes_ps() {
    constexpr int R1 = plane_lanes_r1<N>(), G = N / R1, H = N / 2 + 1;
    constexpr int EX = R1 * (G + 1) > N + 2 ? R1 * (G + 1) : N + 2;
    constexpr int NEED = H > (EX + 1) / 2 ? H : (EX + 1) / 2;
    return NEED + ((12 - NEED % 8) % 8);
}
template <int N> __host__ __device__ constexpr size_t plane_lanes_smem_bytes() {
    return sizeof(float2) * ((size_t)N + (size_t)N * plane_lanes_ps<N>());
}

template <int N, int IN>
__global__ void __launch_bounds__(plane_lanes_threads<N>()) k_plane_r2c_lanes(RowR2CArgs a) {
    constexpr int NT = plane_lanes_threads<N>(), R1 = plane_lanes_r1<N>(), G = N / R1, XS = G + 1;
    constexpr int H = N / 2 + 1, NRP = nrp_of(N), P = N / 2, PS = plane_lanes_ps<N>(), PW = 32 / G;
    constexpr int J = (R1 + G - 1) / G, M = (H + G - 1) / G;
    static_assert(IN == ROW_IN_I64 || IN == ROW_IN_F32, "grid or float input");
    static_assert(P % PW == 0 && 32 % G == 0, "whole lane groups");
    extern __shared__ float4 smem_raw[];
    float2* tw = reinterpret_cast<float2*>(smem_raw);
    float2* pl = tw + N;
    const int x = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane / G, q = lane % G;
    for (int i = threadIdx.x; i < N; i += NT) tw[i] = a.tw[i];
    float scale = 1.0f;
    unsigned cur = 0;
    if constexpr (IN == ROW_IN_I64) {
        const double S = a.slot_S[a.slot];
        const long long tot = a.slot_total[a.slot];
        scale = a.bf16 ? (tot > 0 ? (float)(1.0 / (double)tot) : 0.0f) : (float)S;
        if (a.rowstamp) cur = *a.stamp;
    }
    // the stamps of this group's rows 2u, 2u + 1, loaded one pair ahead
    unsigned sa = 0, sb = 0;
    if constexpr (IN == ROW_IN_I64) {
        const int u = warp * PW + grp;
        if (a.rowstamp && u < P) {
            sa = a.rowstamp[(long long)x * N + 2 * u];
            sb = a.rowstamp[(long long)x * N + 2 * u + 1];
        }
    }
    __syncthreads();
    for (int u0 = warp * PW; u0 < P; u0 += (NT / 32) * PW) {
        const int u = u0 + grp;
        float2* ex = pl + (2 * u) * PS; // this pair's two rows
        const long long ra = ((long long)x * N + 2 * u) * N, rb = ra + N;
        float2 v[16];
        if constexpr (IN == ROW_IN_I64) {
            if (a.rowstamp) {
                // rows without a share of this push: zero half spectra, when
                // all of the warp's pairs are such (the warp stays converged)
                const bool mine = sa == cur || sb == cur;
                const int un = u + (NT / 32) * PW;
                sa = un < P ? a.rowstamp[(long long)x * N + 2 * un] : 0u;
                sb = un < P ? a.rowstamp[(long long)x * N + 2 * un + 1] : 0u;
                if (!__any_sync(0xffffffffu, mine)) {
#pragma unroll
                    for (int m = 0; m < M; ++m) {
                        const int k = q + G * m;
                        if (k < H) {
                            ex[k] = make_float2(0.f, 0.f);
                            ex[PS + k] = make_float2(0.f, 0.f);
                        }
                    }
                    continue;
                }
            }
            long long xa[R1], xb[R1];
#pragma unroll
            for (int p = 0; p < R1; ++p) {
                xa[p] = a.grid[ra + q + G * p];
                xb[p] = a.grid[rb + q + G * p];
            }
#pragma unroll
            for (int p = 0; p < R1; ++p) v[p] = make_float2(__ll2float_rn(xa[p]) * scale, __ll2float_rn(xb[p]) * scale);
        } else {
#pragma unroll
            for (int p = 0; p < R1; ++p) v[p] = make_float2(a.fin[ra + q + G * p], a.fin[rb + q + G * p]);
        }
        dft<R1, -1>(v);
#pragma unroll
        for (int k1 = 1; k1 < R1; ++k1) v[k1] = cmul(v[k1], tw[q * k1]);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) ex[k1 * XS + q] = v[k1];
        __syncwarp();
        float2 z[J * G];
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int k1 = q + G * j;
            if (k1 < R1) {
                float2 w[G];
#pragma unroll
                for (int r = 0; r < G; ++r) w[r] = ex[k1 * XS + r];
                dft<G, -1>(w);
#pragma unroll
                for (int k2 = 0; k2 < G; ++k2) z[j * G + k2] = w[k2];
            }
        }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int k1 = q + G * j;
            if (k1 < R1) {
#pragma unroll
                for (int k2 = 0; k2 < G; ++k2) ex[k1 + R1 * k2] = z[j * G + k2]; // Z in natural order
            }
        }
        __syncwarp();
        // X_a = (Z_k + conj Z_{N-k}) / 2, X_b = (Z_k - conj Z_{N-k}) / (2 i)
        float2 ua[M], ub[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int k = q + G * m;
            if (k < H) {
                const float2 zk = ex[k], zn = ex[k == 0 ? 0 : N - k];
                ua[m] = make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
                ub[m] = make_float2(0.5f * (zk.y + zn.y), 0.5f * (zn.x - zk.x));
            }
        }
        __syncwarp();
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int k = q + G * m;
            if (k < H) {
                ex[k] = ua[m];      // row 2u
                ex[PS + k] = ub[m]; // row 2u + 1
            }
        }
    }
    __syncthreads();
    for (int it = threadIdx.x; it < H * G; it += NT) {
        int c, r;
        plane_item<N>(it, G, c, r);
        float2 v[16];
#pragma unroll
        for (int p = 0; p < R1; ++p) v[p] = pl[(r + G * p) * PS + c];
        dft<R1, -1>(v);
#pragma unroll
        for (int k1 = 1; k1 < R1; ++k1) v[k1] = cmul(v[k1], tw[r * k1]);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) pl[(k1 * G + r) * PS + c] = v[k1]; // the rows it read
    }
    __syncthreads();
    for (int it = threadIdx.x; it < H * R1; it += NT) {
        int c, k1;
        plane_item<N>(it, R1, c, k1);
        float2 w[G];
#pragma unroll
        for (int r = 0; r < G; ++r) w[r] = pl[(k1 * G + r) * PS + c];
        dft<G, -1>(w);
#pragma unroll
        for (int k2 = 0; k2 < G; ++k2) a.dst[((long long)x * N + (k1 + R1 * k2)) * NRP + c] = w[k2];
    }
}

// Inverse of k_plane_r2c_lanes for one x-plane: y inverse with item (c, r)
// taking its R1 inputs straight from global memory, the second stage in
// place (its outputs Y[k1 + R1 k2] land on the rows k1 G + k2 it read, so
// no item overwrites another's input), then the z inverse per row pair
// (real rows 2u, 2u + 1 as one complex transform, Hermitian-extended), the
// pair's exchange on the two plane rows that held its input, and the
// results (times `scale`) written from registers.
template <int N>
__global__ void __launch_bounds__(plane_lanes_threads<N>()) k_plane_c2r_lanes(RowC2RArgs a) {
    constexpr int NT = plane_lanes_threads<N>(), R1 = plane_lanes_r1<N>(), G = N / R1, XS = G + 1;
    constexpr int H = N / 2 + 1, NRP = nrp_of(N), P = N / 2, PS = plane_lanes_ps<N>(), PW = 32 / G;
    constexpr int J = (R1 + G - 1) / G;
    static_assert(P % PW == 0 && 32 % G == 0, "whole lane groups");
    if (blockIdx.x >= N) {
        plane_near_ctas<N, NT>(a.near);
        return;
    }
    extern __shared__ float4 smem_raw[];
    float2* tw = reinterpret_cast<float2*>(smem_raw);
    float2* pl = tw + N;
    const int x = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane / G, q = lane % G;
    for (int i = threadIdx.x; i < N; i += NT) tw[i] = a.tw[i];
    __syncthreads();
    for (int it = threadIdx.x; it < H * G; it += NT) {
        int c, r;
        plane_item<N>(it, G, c, r);
        float2 v[16];
#pragma unroll
        for (int p = 0; p < R1; ++p) v[p] = a.src[((long long)x * N + (r + G * p)) * NRP + c];
        dft<R1, 1>(v);
#pragma unroll
        for (int k1 = 1; k1 < R1; ++k1) {
            float2 w = tw[r * k1];
            w.y = -w.y;
            v[k1] = cmul(v[k1], w);
        }
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) pl[(k1 * G + r) * PS + c] = v[k1];
    }
    __syncthreads();
    for (int it = threadIdx.x; it < H * R1; it += NT) {
        int c, k1;
        plane_item<N>(it, R1, c, k1);
        float2 w[G];
#pragma unroll
        for (int r = 0; r < G; ++r) w[r] = pl[(k1 * G + r) * PS + c];
        dft<G, 1>(w);
#pragma unroll
        for (int k2 = 0; k2 < G; ++k2) pl[(k1 * G + k2) * PS + c] = w[k2]; // Y[k1 + R1 k2]
    }
    __syncthreads();
    static_assert(R1 % 2 == 0 && P == G * (R1 / 2), "pairs as (residue, block)");
    for (int u0 = warp * PW; u0 < P; u0 += (NT / 32) * PW) {
        // group T takes pair u = (T mod G) R1/2 + T / G: the lane groups of a
        // warp then read plane rows one apart (rows (y mod R1) G + y / R1), not
        // 16 apart, which would put all of them on the same banks
        const int T = u0 + grp;
        const int u = (T % G) * (R1 / 2) + T / G;
        // the plane rows of y = 2u and 2u + 1
        float2* xa = pl + (((2 * u) % R1) * G + (2 * u) / R1) * PS;
        float2* xb = pl + (((2 * u + 1) % R1) * G + (2 * u + 1) / R1) * PS;
        // Z_n = X_a(n) + i X_b(n), with X(N - n) = conj X(n) beyond N/2
        float2 v[16];
#pragma unroll
        for (int p = 0; p < R1; ++p) {
            const int n = q + G * p;
            if (n < H) {
                float2 A = xa[n], B = xb[n];
                if (n == 0 || n == N / 2) {
                    A.y = 0.f;
                    B.y = 0.f;
                }
                v[p] = make_float2(A.x - B.y, A.y + B.x);
            } else {
                const float2 A = xa[N - n], B = xb[N - n];
                v[p] = make_float2(A.x + B.y, B.x - A.y);
            }
        }
        __syncwarp(); // every lane of the group has read the pair's rows
        dft<R1, 1>(v);
#pragma unroll
        for (int k1 = 1; k1 < R1; ++k1) {
            float2 w = tw[q * k1];
            w.y = -w.y;
            v[k1] = cmul(v[k1], w);
        }
        // exchange on the pair's two rows: element e at xa[e] (e < PS) or xb[e - PS]
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
            const int e = k1 * XS + q;
            (e < PS ? xa[e] : xb[e - PS]) = v[k1];
        }
        __syncwarp();
        float* oa = a.out + ((long long)x * N + 2 * u) * N;
        float* ob = oa + N;
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int k1 = q + G * j;
            if (k1 < R1) {
                float2 w[G];
#pragma unroll
                for (int r = 0; r < G; ++r) {
                    const int e = k1 * XS + r;
                    w[r] = e < PS ? xa[e] : xb[e - PS];
                }
                dft<G, 1>(w);
#pragma unroll
                for (int k2 = 0; k2 < G; ++k2) {
                    oa[k1 + R1 * k2] = w[k2].x * a.scale;
                    ob[k1 + R1 * k2] = w[k2].y * a.scale;
                }
            }
        }
    }
}

// ------------------------------------------------------------------------
// N = 256: z and y per x-plane on a cluster of C = 4 CTAs.  The 256 x 129
// half plane (264 KB) does not fit one CTA's shared memory, so each x-plane
// goes to a cluster, and the z pass, the y pass and the transposition
// between them stay on chip.  Rank c keeps the y-pass columns kz in
// [CW c, CW c + CW) (CW = N / 2C; rank 0 also the Nyquist column N/2) of all
// N rows in a buffer B[y][PS].
//   forward: rank c transforms rows y in [R c, R c + R) (R = N / C) along z,
//     a row pair per lane group as k_rows_r2c_lanes, and stores each
//     unpacked value in the buffer of the rank that owns its kz, its own or a
//     peer's (distributed shared memory); after the cluster barrier it runs
//     the y pass of its columns as k_plane_r2c_lanes (R1 = G = 16) and writes
//     them out.
//   inverse: rank c runs the y pass of its columns from global memory, the
//     result Y[k1 + 16 k2] on buffer row 16 k1 + k2; after the cluster
//     barrier it transforms rows [R c, R c + R) along z as k_rows_c2r_lanes,
//     reading each kz from the buffer that holds it, and a second barrier
//     keeps every buffer until the peers have read it.
// Two 288-thread CTAs per SM (112 KB of shared memory each), so that one
// CTA's transfers overlap the other's arithmetic.  (Clusters of two, one
// 544-thread CTA per SM with 215 KB, and of eight, three 256-thread CTAs per
// SM with 59 KB, were slower at 256^3: the more CTAs a cluster holds, the
// more of them wait at each barrier for the slowest.)
template <int N> __host__ __device__ constexpr bool plane_cl_ok() { return N == 256; }
constexpr int kPlaneClC = 4, kPlaneClThreads = 288;
template <int N> __host__ __device__ constexpr int plane_cl_ps() { return N / (2 * kPlaneClC) + 4; }
template <int N> __host__ __device__ constexpr size_t plane_cl_smem_bytes() {
    return sizeof(float2) * ((size_t)N + (size_t)N * plane_cl_ps<N>() +
                             (size_t)(kPlaneClThreads / (N / lanes_r1<N>(0))) * rows_lanes_ex<N>());
}
// the rank holding column k of the half spectrum (CW columns a rank, the
// Nyquist column N/2 = C CW on rank 0), its column index there, and back
__device__ __forceinline__ int plane_cl_owner(int k, int CW, int C) { return k == C * CW ? 0 : k / CW; }
__device__ __forceinline__ int plane_cl_col(int k, int CW, int C) { return k == C * CW ? CW : k % CW; }
__device__ __forceinline__ int plane_cl_kz(int rank, int c, int CW, int C) { return c == CW ? C * CW : rank * CW + c; }
// item `it` of a y stage over a rank's columns (CW regular ones, row by row,
// then rank 0's Nyquist column c = CW)
__device__ __forceinline__ void plane_cl_item(int it, int rows, int CW, int& c, int& r) {
    if (it < CW * rows) {
        c = it % CW;
        r = it / CW;
    } else {
        c = CW;
        r = it - CW * rows;
    }
}
// store v at float2 index idx of rank o's buffer (sB: this CTA's buffer as a
// shared::cta address)
__device__ __forceinline__ void plane_cl_put(float2* B, unsigned sB, int rank, int o, int idx, float2 v) {
    if (o == rank) B[idx] = v;
    else cluster_st(cluster_map(sB + 8u * (unsigned)idx, (unsigned)o), v);
}
__device__ __forceinline__ float2 plane_cl_get(const float2* B, unsigned sB, int rank, int o, int idx) {
    return o == rank ? B[idx] : cluster_ld(cluster_map(sB + 8u * (unsigned)idx, (unsigned)o));
}

template <int N, int IN>
__global__ void __cluster_dims__(kPlaneClC, 1, 1) __launch_bounds__(kPlaneClThreads, 2) k_plane_cl_r2c(RowR2CArgs a) {
    constexpr int C = kPlaneClC, NT = kPlaneClThreads, R1 = lanes_r1<N>(0), G = N / R1, PW = 32 / G, H = N / 2 + 1;
    constexpr int NRP = nrp_of(N), PS = plane_cl_ps<N>(), EX = rows_lanes_ex<N>(), CW = N / (2 * C), R = N / C;
    static_assert(R1 == 16 && G == 16 && PW == 2, "16 x 16 rows, two row pairs per warp");
    static_assert(IN == ROW_IN_I64 || IN == ROW_IN_F32, "grid or float input");
    extern __shared__ float4 smem_raw[];
    float2* tw = reinterpret_cast<float2*>(smem_raw);
    float2* B = tw + N;
    const unsigned sB = smem_u32(B);
    const int rank = (int)cluster_rank(), x = blockIdx.x / C;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane / G, q = lane % G;
    float2* ex = B + N * PS + (warp * PW + grp) * EX;
    for (int i = threadIdx.x; i < N; i += NT) tw[i] = a.tw[i];
    float scale = 1.0f;
    unsigned cur = 0;
    if constexpr (IN == ROW_IN_I64) {
        const double S = a.slot_S[a.slot];
        const long long tot = a.slot_total[a.slot];
        scale = a.bf16 ? (tot > 0 ? (float)(1.0 / (double)tot) : 0.0f) : (float)S;
        if (a.rowstamp) cur = *a.stamp;
    }
    // the stamps of this group's rows, loaded one pair ahead
    unsigned sa = 0, sb = 0;
    if constexpr (IN == ROW_IN_I64) {
        const int ya = R * rank + 2 * (warp * PW + grp);
        if (a.rowstamp && warp * PW < R / 2) {
            sa = a.rowstamp[(long long)x * N + ya];
            sb = a.rowstamp[(long long)x * N + ya + 1];
        }
    }
    cluster_sync(); // the peers run (their buffers may be written) and the twiddles are in place
    for (int u0 = warp * PW; u0 < R / 2; u0 += (NT / 32) * PW) {
        const int ya = R * rank + 2 * (u0 + grp), yb = ya + 1;
        const long long ra = ((long long)x * N + ya) * N, rb = ra + N;
        bool zero = false;
        if constexpr (IN == ROW_IN_I64) {
            if (a.rowstamp) {
                // no row of the warp's two pairs holds a share of this push
                const bool mine = sa == cur || sb == cur;
                const int un = u0 + (NT / 32) * PW, yn = R * rank + 2 * (un + grp);
                sa = un < R / 2 ? a.rowstamp[(long long)x * N + yn] : 0u;
                sb = un < R / 2 ? a.rowstamp[(long long)x * N + yn + 1] : 0u;
                zero = !__any_sync(0xffffffffu, mine);
            }
        }
        if (zero) {
#pragma unroll
            for (int m = 0; m < (H + G - 1) / G; ++m) {
                const int k = q + G * m;
                if (k < H) {
                    const int o = plane_cl_owner(k, CW, C), c = plane_cl_col(k, CW, C);
                    plane_cl_put(B, sB, rank, o, ya * PS + c, make_float2(0.f, 0.f));
                    plane_cl_put(B, sB, rank, o, yb * PS + c, make_float2(0.f, 0.f));
                }
            }
            continue;
        }
        float2 v[16];
        if constexpr (IN == ROW_IN_I64) {
            long long xa[R1], xb[R1];
#pragma unroll
            for (int p = 0; p < R1; ++p) {
                xa[p] = a.grid[ra + q + G * p];
                xb[p] = a.grid[rb + q + G * p];
            }
            if (a.zero_in) {
                long long* g = const_cast<long long*>(a.grid);
#pragma unroll
                for (int p = 0; p < R1; ++p) {
                    g[ra + q + G * p] = 0;
                    g[rb + q + G * p] = 0;
                }
            }
#pragma unroll
            for (int p = 0; p < R1; ++p) v[p] = make_float2(__ll2float_rn(xa[p]) * scale, __ll2float_rn(xb[p]) * scale);
        } else {
#pragma unroll
            for (int p = 0; p < R1; ++p) v[p] = make_float2(a.fin[ra + q + G * p], a.fin[rb + q + G * p]);
        }
        int t0, ts;
        fft_row_lanes<N, -1>(v, ex, tw, q, t0, ts); // G = 16: every lane active, Z[t0 + ts k] = v[k]
#pragma unroll
        for (int k = 0; k < 16; ++k) ex[t0 + ts * k] = v[k];
        __syncwarp();
        // X_a = (Z_k + conj Z_{N-k}) / 2, X_b = (Z_k - conj Z_{N-k}) / (2 i), to the owner of column k
#pragma unroll
        for (int m = 0; m < (H + G - 1) / G; ++m) {
            const int k = q + G * m;
            if (k < H) {
                const float2 zk = ex[k], zn = ex[k == 0 ? 0 : N - k];
                const int o = plane_cl_owner(k, CW, C), c = plane_cl_col(k, CW, C);
                plane_cl_put(B, sB, rank, o, ya * PS + c, make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y)));
                plane_cl_put(B, sB, rank, o, yb * PS + c, make_float2(0.5f * (zk.y + zn.y), 0.5f * (zn.x - zk.x)));
            }
        }
        __syncwarp(); // the exchange buffer is free for the next pair
    }
    cluster_sync(); // all N rows of this rank's columns are in its buffer
    const int NC = rank ? CW : CW + 1;
    for (int it = threadIdx.x; it < NC * G; it += NT) {
        int c, r;
        plane_cl_item(it, G, CW, c, r);
        float2 v[16];
#pragma unroll
        for (int p = 0; p < R1; ++p) v[p] = B[(r + G * p) * PS + c];
        dft<R1, -1>(v);
#pragma unroll
        for (int k1 = 1; k1 < R1; ++k1) v[k1] = cmul(v[k1], tw[r * k1]);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) B[(k1 * G + r) * PS + c] = v[k1]; // the rows it read
    }
    __syncthreads();
    for (int it = threadIdx.x; it < NC * R1; it += NT) {
        int c, k1;
        plane_cl_item(it, R1, CW, c, k1);
        float2 w[G];
#pragma unroll
        for (int r = 0; r < G; ++r) w[r] = B[(k1 * G + r) * PS + c];
        dft<G, -1>(w);
        const int kz = plane_cl_kz(rank, c, CW, C);
#pragma unroll
        for (int k2 = 0; k2 < G; ++k2) a.dst[((long long)x * N + (k1 + R1 * k2)) * NRP + kz] = w[k2];
    }
}

template <int N>
__global__ void __cluster_dims__(kPlaneClC, 1, 1) __launch_bounds__(kPlaneClThreads, 2) k_plane_cl_c2r(RowC2RArgs a) {
    constexpr int C = kPlaneClC, NT = kPlaneClThreads, R1 = lanes_r1<N>(0), G = N / R1, PW = 32 / G, H = N / 2 + 1;
    constexpr int NRP = nrp_of(N), PS = plane_cl_ps<N>(), EX = rows_lanes_ex<N>(), CW = N / (2 * C), R = N / C;
    static_assert(R1 == 16 && G == 16 && PW == 2, "16 x 16 rows, two row pairs per warp");
    static_assert(2 * H <= EX, "both half spectra fit the exchange buffer");
    if (blockIdx.x >= C * N) {
        // whole clusters past the planes: the near-field list (no cluster barrier)
        plane_near_ctas<N, NT, C * N>(a.near);
        return;
    }
    extern __shared__ float4 smem_raw[];
    float2* tw = reinterpret_cast<float2*>(smem_raw);
    float2* B = tw + N;
    const unsigned sB = smem_u32(B);
    const int rank = (int)cluster_rank(), x = blockIdx.x / C;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane / G, q = lane % G;
    float2* ex = B + N * PS + (warp * PW + grp) * EX;
    for (int i = threadIdx.x; i < N; i += NT) tw[i] = a.tw[i];
    __syncthreads();
    const int NC = rank ? CW : CW + 1;
    for (int it = threadIdx.x; it < NC * G; it += NT) {
        int c, r;
        plane_cl_item(it, G, CW, c, r);
        const int kz = plane_cl_kz(rank, c, CW, C);
        float2 v[16];
#pragma unroll
        for (int p = 0; p < R1; ++p) v[p] = a.src[((long long)x * N + (r + G * p)) * NRP + kz];
        dft<R1, 1>(v);
#pragma unroll
        for (int k1 = 1; k1 < R1; ++k1) {
            float2 w = tw[r * k1];
            w.y = -w.y;
            v[k1] = cmul(v[k1], w);
        }
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) B[(k1 * G + r) * PS + c] = v[k1];
    }
    __syncthreads();
    for (int it = threadIdx.x; it < NC * R1; it += NT) {
        int c, k1;
        plane_cl_item(it, R1, CW, c, k1);
        float2 w[G];
#pragma unroll
        for (int r = 0; r < G; ++r) w[r] = B[(k1 * G + r) * PS + c];
        dft<G, 1>(w);
#pragma unroll
        for (int k2 = 0; k2 < G; ++k2) B[(k1 * G + k2) * PS + c] = w[k2]; // Y[k1 + R1 k2]
    }
    cluster_sync(); // every rank's y results are visible in the cluster
    for (int u0 = warp * PW; u0 < R / 2; u0 += (NT / 32) * PW) {
        const int ya = R * rank + 2 * (u0 + grp), yb = ya + 1;
        // buffer rows of y = k1 + R1 k2: G k1 + k2
        const int ba = (ya % R1) * G + ya / R1, bb = (yb % R1) * G + yb / R1;
        float2* xa = ex;
        float2* xb = ex + H;
#pragma unroll
        for (int m = 0; m < (H + G - 1) / G; ++m) {
            const int k = q + G * m;
            if (k < H) {
                const int o = plane_cl_owner(k, CW, C), c = plane_cl_col(k, CW, C);
                float2 A = plane_cl_get(B, sB, rank, o, ba * PS + c);
                float2 Bv = plane_cl_get(B, sB, rank, o, bb * PS + c);
                if (k == 0 || k == N / 2) {
                    A.y = 0.f;
                    Bv.y = 0.f;
                }
                xa[k] = A;
                xb[k] = Bv;
            }
        }
        __syncwarp();
        // Z_n = X_a(n) + i X_b(n), with the Hermitian extension X(N - k) = conj X(k)
        float2 v[16];
#pragma unroll
        for (int p = 0; p < R1; ++p) {
            const int n = q + G * p;
            if (n < H) {
                const float2 A = xa[n], Bv = xb[n];
                v[p] = make_float2(A.x - Bv.y, A.y + Bv.x);
            } else {
                const float2 A = xa[N - n], Bv = xb[N - n];
                v[p] = make_float2(A.x + Bv.y, Bv.x - A.y);
            }
        }
        __syncwarp();
        int t0, ts;
        fft_row_lanes<N, 1>(v, ex, tw, q, t0, ts);
        float* oa = a.out + ((long long)x * N + ya) * N;
        float* ob = oa + N;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            oa[t0 + ts * k] = v[k].x * a.scale;
            ob[t0 + ts * k] = v[k].y * a.scale;
        }
    }
    cluster_sync(); // the peers have read this rank's buffer
}

// ------------------------------------------------------------------------
// Host-side launchers for one N.
struct MacArgs;
struct FftOps {
    int n;
    cudaError_t (*init)();
    void (*rows_r2c)(const RowR2CArgs&, cudaStream_t);
    void (*cols)(const ColArgs&, cudaStream_t);
    void (*rows_c2r)(const RowC2RArgs&, cudaStream_t);
    // z + y in one kernel per x-plane (null where the half plane does not fit)
    void (*plane_r2c)(const RowR2CArgs&, cudaStream_t);
    void (*plane_c2r)(const RowC2RArgs&, cudaStream_t);
    // fused TMA shell MAC over the full tiles (null where not built), FP32 / BF16 ring
    void (*mac_f32)(const MacArgs&, cudaStream_t);
    void (*mac_bf16)(const MacArgs&, cudaStream_t);
    // warp-specialised MAC over every tile, Nyquist ones included (null where
    // not built): one tile per CTA, or the tiles of lines q and N - q together
    void (*mac_ws_f32)(const MacArgs&, cudaStream_t);
    void (*mac_ws_bf16)(const MacArgs&, cudaStream_t);
    void (*mac_ws2_f32)(const MacArgs&, cudaStream_t);
    void (*mac_ws2_bf16)(const MacArgs&, cudaStream_t);
    int full_tiles; // tiles of the full 16-column chunks (the Nyquist tiles follow)
    // the y / x pass kernel of grids with more than one: FFT_COLS_STAGES
    // (block-wide Stockham stages), FFT_COLS_LANES (one lane per column, four
    // tile stages, one CTA per SM), FFT_COLS_LANES3 (three stages, two CTAs
    // per SM), FFT_COLS_TMA (the tiles moved by tensor-map TMA, three stages,
    // two CTAs per SM) or FFT_COLS_TMA4 (TMA, four stages, one CTA per SM);
    // chosen by the autotuner or LC_FFT_VARIANT, shared by the process
    int (*cols_variants)();          // bit mask of the variants built for this N
    void (*set_cols_variant)(int);
    int (*cols_variant)();
    // extra CTAs of plane_c2r for a near-field list of `items` items on a GPU
    // of nsm SMs (0: run the list in a launch of its own)
    int (*plane_near_ctas)(long long items, int nsm);
    // whether the per-step transforms take plane_r2c / plane_c2r now (always
    // where plane_r2c exists for one CTA per plane; for N = 256 with the
    // FFT_PLANE4 form); plane_clustered: a cluster of CTAs per plane
    // (N = 256), whose plane kernels take grid or float input only
    bool (*plane_on)();
    bool plane_clustered;
};
// FFT_PLANE4 (N = 256): z and y per x-plane on a cluster of four CTAs
// (k_plane_cl_r2c / k_plane_cl_c2r), the x passes in the FFT_COLS_LANES form
enum {
    FFT_COLS_STAGES = 0,
    FFT_COLS_LANES = 1,
    FFT_COLS_LANES3 = 2,
    FFT_COLS_TMA = 3,
    FFT_COLS_TMA4 = 4,
    FFT_PLANE4 = 5,
    FFT_NVAR = 6
};

template <int N> struct Launch {
    static constexpr int CW = cw_of(N), NCH = (N / 2) / CW;
    static int col_tiles() { return N * NCH + N / CW; }
    // the SM count, read once per process
    static int sms() {
        static int n = 0;
        if (!n) {
            int dev = 0;
            cudaGetDevice(&dev);
            if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
                cudaGetLastError();
                n = 148;
            }
        }
        return n;
    }
    // CTAs of a persistent row pass: 4 per SM
    static int pp_ctas() { return 4 * sms(); }
    // the pipelined column pass (N >= 256) or the register-prefetch one
    static constexpr bool kColsPl = N >= 256;
    // CTAs of the pipelined column pass: as many as fit on the device at once
    template <int DIR, int OUT> static int cols_pl_ctas() {
        static int ctas = 0;
        if (!ctas) {
            int occ = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cols_pl<N, DIR, OUT>, cols_pl_threads(N),
                                                              cols_pl_smem_bytes<N>()) != cudaSuccess || occ <= 0) {
                cudaGetLastError();
                occ = 1;
            }
            ctas = occ * sms();
        }
        return ctas;
    }
    static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
    // the column-pass variant in use (FFT_COLS_*)
    // (grids with plane kernels: FFT_COLS_STAGES = the staged plane kernels,
    // FFT_COLS_LANES = k_plane_r2c_lanes / k_plane_c2r_lanes)
    static int& variant() {
        static int v = (cols_lanes_ok<N>() || plane_lanes_ok<N>()) ? FFT_COLS_LANES : FFT_COLS_STAGES;
        return v;
    }
    static int variants_built() {
        return (1 << FFT_COLS_STAGES) |
               (cols_lanes_ok<N>()
                    ? (1 << FFT_COLS_LANES) | (1 << FFT_COLS_LANES3) | (1 << FFT_COLS_TMA) | (1 << FFT_COLS_TMA4)
                    : 0) |
               (plane_lanes_ok<N>() ? (1 << FFT_COLS_LANES) : 0) |
               (plane_cl_ok<N>() ? (1 << FFT_PLANE4) : 0);
    }
    static bool plane_on() {
        if constexpr (plane_ok<N>()) return true;
        else if constexpr (plane_cl_ok<N>()) return variant() == FFT_PLANE4;
        else return false;
    }
    static void set_variant(int v) {
        if (v >= 0 && v < FFT_NVAR && (variants_built() >> v & 1)) variant() = v;
    }
    static int get_variant() { return variant(); }
    template <int DIR, int OUT, int S> static int cols_lanes_ctas() {
        static int ctas = 0;
        if (!ctas) {
            int occ = 0;
            if constexpr (cols_lanes_ok<N>()) {
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cols_lanes<N, DIR, OUT, S>,
                                                                  cols_lanes_threads(),
                                                                  cols_lanes_smem_bytes<N, S>()) != cudaSuccess ||
                    occ <= 0) {
                    cudaGetLastError();
                    occ = 1;
                }
            }
            ctas = (occ > 0 ? occ : 1) * sms();
        }
        return ctas;
    }
    template <int DIR, int OUT, int S> static void cols_lanes_launch(const ColArgs& a, int ntiles, cudaStream_t st) {
        if constexpr (cols_lanes_ok<N>()) {
            const int c = cols_lanes_ctas<DIR, OUT, S>();
            launch_k(k_cols_lanes<N, DIR, OUT, S>, dim3((unsigned)(ntiles < c ? ntiles : c)), cols_lanes_threads(),
                     cols_lanes_smem_bytes<N, S>(), st, a, ntiles);
        }
    }
    static bool lanes_form() { return variant() != FFT_COLS_STAGES; }
    template <int DIR, int OUT, int S> static void cols_tma_launch(const ColArgs& a, int ntiles, cudaStream_t st) {
        if constexpr (cols_lanes_ok<N>()) {
            static int ctas = 0;
            if (!ctas) {
                int occ = 0;
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cols_tma<N, DIR, OUT, S>, cols_lanes_threads(),
                                                                  cols_tma_smem_bytes<N, S>()) != cudaSuccess ||
                    occ <= 0) {
                    cudaGetLastError();
                    occ = 1;
                }
                ctas = occ * sms();
            }
            launch_k(k_cols_tma<N, DIR, OUT, S>, dim3((unsigned)(ntiles < ctas ? ntiles : ctas)), cols_lanes_threads(),
                     cols_tma_smem_bytes<N, S>(), st, a, ntiles, *a.tmap);
        }
    }
    template <int DIR, int OUT> static void cols_plain(const ColArgs& a, int ntiles, cudaStream_t st) {
        if constexpr (cols_lanes_ok<N>()) {
            if ((variant() == FFT_COLS_TMA || variant() == FFT_COLS_TMA4) && a.tmap) {
                if (variant() == FFT_COLS_TMA4) cols_tma_launch<DIR, OUT, 4>(a, ntiles, st);
                else cols_tma_launch<DIR, OUT, 3>(a, ntiles, st);
                return;
            }
            if (lanes_form() && aligned16(a.src)) {
                if (variant() == FFT_COLS_LANES3) cols_lanes_launch<DIR, OUT, 3>(a, ntiles, st);
                else cols_lanes_launch<DIR, OUT, 4>(a, ntiles, st);
                return;
            }
        }
        if constexpr (kColsPl) {
            if (aligned16(a.src)) { // 16-byte copies need a 16-byte aligned source
                const int c = cols_pl_ctas<DIR, OUT>();
                launch_k(k_cols_pl<N, DIR, OUT>, dim3((unsigned)(ntiles < c ? ntiles : c)), cols_pl_threads(N),
                         cols_pl_smem_bytes<N>(), st, a, ntiles);
                return;
            }
        }
        // persistent: a few CTAs per SM, each walking tiles
        launch_k(k_cols_pp<N, DIR, OUT>, dim3((unsigned)(ntiles < pp_ctas() ? ntiles : pp_ctas())), col_threads_of(N),
                 cols_smem_bytes<N>(), st, a, ntiles);
    }
    static long long row_blocks() { return ((long long)N * N + 2 * row_pairs_of(N) - 1) / (2 * row_pairs_of(N)); }

    static cudaError_t init() {
        cudaError_t e = cudaSuccess;
        const int cs = (int)cols_smem_bytes<N>(), rs = (int)rows_smem_bytes<N>();
#define LC_ATTR(K, S) \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, S)
        LC_ATTR((k_rows_r2c<N, ROW_IN_I64>), rs);
        LC_ATTR((k_rows_r2c<N, ROW_IN_F32>), rs);
        LC_ATTR((k_rows_r2c<N, ROW_IN_WEDGE>), rs);
        LC_ATTR((k_rows_c2r<N>), rs);
        if constexpr (kRowsPl) {
            const int r64 = (int)rows_r2c_pl_smem_bytes<N, ROW_IN_I64>(), r32 = (int)rows_r2c_pl_smem_bytes<N, ROW_IN_F32>();
            LC_ATTR((k_rows_r2c_pl<N, ROW_IN_I64>), r64);
            LC_ATTR((k_rows_r2c_pl<N, ROW_IN_F32>), r32);
            LC_ATTR((k_rows_c2r_pl<N>), (int)rows_c2r_pl_smem_bytes<N>());
        }
        if constexpr (kColsPl) {
            const int ps2 = (int)cols_pl_smem_bytes<N>();
            LC_ATTR((k_cols_pl<N, -1, COL_OUT_PLAIN>), ps2);
            LC_ATTR((k_cols_pl<N, -1, COL_OUT_BF16>), ps2);
            LC_ATTR((k_cols_pl<N, -1, COL_OUT_WEDGE>), ps2);
            LC_ATTR((k_cols_pl<N, -1, COL_OUT_RING_F32>), ps2);
            LC_ATTR((k_cols_pl<N, 1, COL_OUT_PLAIN>), ps2);
            if constexpr (rows_lanes_ok<N>()) {
                const int rl = (int)rows_lanes_smem_bytes<N>();
                LC_ATTR((k_rows_r2c_lanes<N, ROW_IN_I64>), rl);
                LC_ATTR((k_rows_r2c_lanes<N, ROW_IN_F32>), rl);
                LC_ATTR((k_rows_c2r_lanes<N>), rl);
            }
            if constexpr (cols_lanes_ok<N>()) {
                const int l4 = (int)cols_lanes_smem_bytes<N, 4>(), l3 = (int)cols_lanes_smem_bytes<N, 3>();
                LC_ATTR((k_cols_lanes<N, -1, COL_OUT_PLAIN, 4>), l4);
                LC_ATTR((k_cols_lanes<N, -1, COL_OUT_BF16, 4>), l4);
                LC_ATTR((k_cols_lanes<N, -1, COL_OUT_WEDGE, 4>), l4);
                LC_ATTR((k_cols_lanes<N, -1, COL_OUT_RING_F32, 4>), l4);
                LC_ATTR((k_cols_lanes<N, 1, COL_OUT_PLAIN, 4>), l4);
                LC_ATTR((k_cols_lanes<N, -1, COL_OUT_PLAIN, 3>), l3);
                LC_ATTR((k_cols_lanes<N, -1, COL_OUT_BF16, 3>), l3);
                LC_ATTR((k_cols_lanes<N, -1, COL_OUT_WEDGE, 3>), l3);
                LC_ATTR((k_cols_lanes<N, -1, COL_OUT_RING_F32, 3>), l3);
                LC_ATTR((k_cols_lanes<N, 1, COL_OUT_PLAIN, 3>), l3);
                const int tm = (int)cols_tma_smem_bytes<N, 3>(), t4 = (int)cols_tma_smem_bytes<N, 4>();
                LC_ATTR((k_cols_tma<N, -1, COL_OUT_PLAIN, 3>), tm);
                LC_ATTR((k_cols_tma<N, -1, COL_OUT_BF16, 3>), tm);
                LC_ATTR((k_cols_tma<N, -1, COL_OUT_WEDGE, 3>), tm);
                LC_ATTR((k_cols_tma<N, -1, COL_OUT_RING_F32, 3>), tm);
                LC_ATTR((k_cols_tma<N, 1, COL_OUT_PLAIN, 3>), tm);
                LC_ATTR((k_cols_tma<N, -1, COL_OUT_PLAIN, 4>), t4);
                LC_ATTR((k_cols_tma<N, -1, COL_OUT_BF16, 4>), t4);
                LC_ATTR((k_cols_tma<N, -1, COL_OUT_WEDGE, 4>), t4);
                LC_ATTR((k_cols_tma<N, -1, COL_OUT_RING_F32, 4>), t4);
                LC_ATTR((k_cols_tma<N, 1, COL_OUT_PLAIN, 4>), t4);
            }
        } else {
            LC_ATTR((k_cols_pp<N, -1, COL_OUT_PLAIN>), cs);
            LC_ATTR((k_cols_pp<N, -1, COL_OUT_BF16>), cs);
            LC_ATTR((k_cols_pp<N, -1, COL_OUT_WEDGE>), cs);
            LC_ATTR((k_cols_pp<N, -1, COL_OUT_RING_F32>), cs);
            LC_ATTR((k_cols_pp<N, 1, COL_OUT_PLAIN>), cs);
        }
        LC_ATTR((k_cols<N, 1, COL_IN_MAC_F32, COL_OUT_PLAIN>), cs);
        LC_ATTR((k_cols<N, 1, COL_IN_MAC_BF16, COL_OUT_PLAIN>), cs);
        if constexpr (!kColsPl) {
            LC_ATTR((k_cols<N, 1, COL_IN_MAC_F32_X, COL_OUT_PLAIN>), cs);
            LC_ATTR((k_cols<N, 1, COL_IN_MAC_BF16_X, COL_OUT_PLAIN>), cs);
        }
        if constexpr (plane_ok<N>()) {
            const int ps = (int)plane_smem_bytes<N>();
            LC_ATTR((k_plane_r2c<N, ROW_IN_I64>), ps);
            LC_ATTR((k_plane_r2c<N, ROW_IN_F32>), ps);
            LC_ATTR((k_plane_r2c<N, ROW_IN_WEDGE>), ps);
            LC_ATTR((k_plane_c2r<N>), ps);
        }
        if constexpr (plane_lanes_ok<N>()) {
            const int pls = (int)plane_lanes_smem_bytes<N>();
            LC_ATTR((k_plane_r2c_lanes<N, ROW_IN_I64>), pls);
            LC_ATTR((k_plane_r2c_lanes<N, ROW_IN_F32>), pls);
            LC_ATTR((k_plane_c2r_lanes<N>), pls);
        }
        if constexpr (plane_cl_ok<N>()) {
            const int pc = (int)plane_cl_smem_bytes<N>();
            LC_ATTR((k_plane_cl_r2c<N, ROW_IN_I64>), pc);
            LC_ATTR((k_plane_cl_r2c<N, ROW_IN_F32>), pc);
            LC_ATTR((k_plane_cl_c2r<N>), pc);
        }
#undef LC_ATTR
        return e;
    }
    static void plane_r2c(const RowR2CArgs& a, cudaStream_t st) {
        if constexpr (plane_ok<N>()) {
            const size_t sm = plane_smem_bytes<N>();
            constexpr int NT = plane_threads_of(N);
            if constexpr (plane_lanes_ok<N>()) {
                if (lanes_form() && a.in_mode != ROW_IN_WEDGE) {
                    constexpr int NL = plane_lanes_threads<N>();
                    const size_t sl = plane_lanes_smem_bytes<N>();
                    if (a.in_mode == ROW_IN_I64) launch_k(k_plane_r2c_lanes<N, ROW_IN_I64>, N, NL, sl, st, a);
                    else launch_k(k_plane_r2c_lanes<N, ROW_IN_F32>, N, NL, sl, st, a);
                    return;
                }
            }
            if (a.in_mode == ROW_IN_I64) launch_k(k_plane_r2c<N, ROW_IN_I64>, N, NT, sm, st, a);
            else if (a.in_mode == ROW_IN_F32) launch_k(k_plane_r2c<N, ROW_IN_F32>, N, NT, sm, st, a);
            else launch_k(k_plane_r2c<N, ROW_IN_WEDGE>, N, NT, sm, st, a);
        } else if constexpr (plane_cl_ok<N>()) {
            // a cluster per x-plane; grid or float input only
            constexpr size_t sm = plane_cl_smem_bytes<N>();
            if (a.in_mode == ROW_IN_I64)
                launch_k(k_plane_cl_r2c<N, ROW_IN_I64>, kPlaneClC * N, kPlaneClThreads, sm, st, a);
            else if (a.in_mode == ROW_IN_F32)
                launch_k(k_plane_cl_r2c<N, ROW_IN_F32>, kPlaneClC * N, kPlaneClThreads, sm, st, a);
        }
    }
    static void plane_c2r(const RowC2RArgs& a, cudaStream_t st) {
        if constexpr (plane_ok<N>()) {
            if constexpr (plane_lanes_ok<N>()) {
                if (lanes_form()) {
                    launch_k(k_plane_c2r_lanes<N>, N + a.near.ctas, plane_lanes_threads<N>(), plane_lanes_smem_bytes<N>(),
                             st, a);
                    return;
                }
            }
            launch_k(k_plane_c2r<N>, N + a.near.ctas, plane_threads_of(N), plane_smem_bytes<N>(), st, a);
        } else if constexpr (plane_cl_ok<N>()) {
            // near.ctas is a multiple of the cluster size: whole clusters
            launch_k(k_plane_cl_c2r<N>, kPlaneClC * N + a.near.ctas, kPlaneClThreads, plane_cl_smem_bytes<N>(), st, a);
        }
    }
    // The near-field list on the SMs the N plane CTAs (one per SM) leave idle
    // in their last wave, about one item a thread, if that leaves at most
    // N / 16 items a thread: the planes' own time grows with N, and the list
    // should end within it.
    // With a cluster per plane, the list takes whole clusters.
    static int plane_near_ctas(long long items, int nsm) {
        int nt = 0, planes = 0, unit = 1, slots = nsm;
        if constexpr (plane_ok<N>()) {
            nt = plane_threads_of(N);
            if constexpr (plane_lanes_ok<N>())
                if (lanes_form()) nt = plane_lanes_threads<N>();
            planes = N;
        } else if constexpr (plane_cl_ok<N>()) {
            unit = kPlaneClC;
            nt = kPlaneClThreads;
            planes = kPlaneClC * N;
            slots = 2 * nsm; // two CTAs resident per SM
        }
        if (planes == 0 || nsm <= 0 || items <= 0) return 0;
        int idle = (planes % slots) ? slots - planes % slots : 0;
        idle -= idle % unit;
        if (idle == 0) return 0;
        long long want = (items + nt - 1) / nt;
        want += (unit - want % unit) % unit;
        const long long c = want < idle ? want : idle;
        return items <= c * nt * (N / 16) ? (int)c : 0;
    }
    static constexpr bool kRowsPl = N >= 256;
    template <class Kern> static int occ_ctas(Kern k, size_t smem) {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kThreads, smem) != cudaSuccess || occ <= 0) {
            cudaGetLastError();
            occ = 1;
        }
        return occ * sms();
    }
    template <class Kern> static int occ_ctas_t(Kern k, int threads, size_t smem) {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, threads, smem) != cudaSuccess || occ <= 0) {
            cudaGetLastError();
            occ = 1;
        }
        return occ * sms();
    }
    static void rows_r2c(const RowR2CArgs& a, cudaStream_t st) {
        const int nb = (int)row_blocks();
        if constexpr (rows_lanes_ok<N>()) {
            if (lanes_form() && (a.in_mode == ROW_IN_I64 || a.in_mode == ROW_IN_F32)) {
                const long long npairs = a.nrows / 2;
                const size_t sm = rows_lanes_smem_bytes<N>();
                if (a.in_mode == ROW_IN_I64) {
                    static const int c = occ_ctas_t(k_rows_r2c_lanes<N, ROW_IN_I64>, kRowsLanesThreads, sm);
                    launch_k(k_rows_r2c_lanes<N, ROW_IN_I64>, dim3((unsigned)c), kRowsLanesThreads, sm, st, a, npairs);
                } else {
                    static const int c = occ_ctas_t(k_rows_r2c_lanes<N, ROW_IN_F32>, kRowsLanesThreads, sm);
                    launch_k(k_rows_r2c_lanes<N, ROW_IN_F32>, dim3((unsigned)c), kRowsLanesThreads, sm, st, a, npairs);
                }
                return;
            }
        }
        if constexpr (kRowsPl) {
            if (a.in_mode == ROW_IN_I64 && !aligned16(a.grid) && a.zero_in) {
                // the register pass does not zero the grid: clear it after
                launch_k(k_rows_r2c<N, ROW_IN_I64>, dim3((unsigned)(nb < pp_ctas() ? nb : pp_ctas())), kThreads,
                         rows_smem_bytes<N>(), st, a, nb);
                cudaMemsetAsync(const_cast<long long*>(a.grid), 0, sizeof(long long) * N * N * N, st);
                return;
            }
            if (a.in_mode == ROW_IN_I64 && aligned16(a.grid)) {
                static const int c = occ_ctas(k_rows_r2c_pl<N, ROW_IN_I64>, rows_r2c_pl_smem_bytes<N, ROW_IN_I64>());
                launch_k(k_rows_r2c_pl<N, ROW_IN_I64>, dim3((unsigned)(nb < c ? nb : c)), kThreads,
                         rows_r2c_pl_smem_bytes<N, ROW_IN_I64>(), st, a, nb);
                return;
            }
            if (a.in_mode == ROW_IN_F32 && aligned16(a.fin)) {
                static const int c = occ_ctas(k_rows_r2c_pl<N, ROW_IN_F32>, rows_r2c_pl_smem_bytes<N, ROW_IN_F32>());
                launch_k(k_rows_r2c_pl<N, ROW_IN_F32>, dim3((unsigned)(nb < c ? nb : c)), kThreads,
                         rows_r2c_pl_smem_bytes<N, ROW_IN_F32>(), st, a, nb);
                return;
            }
        }
        const dim3 g((unsigned)(nb < pp_ctas() ? nb : pp_ctas()));
        const size_t sm = rows_smem_bytes<N>();
        if (a.in_mode == ROW_IN_I64) launch_k(k_rows_r2c<N, ROW_IN_I64>, g, kThreads, sm, st, a, nb);
        else if (a.in_mode == ROW_IN_F32) launch_k(k_rows_r2c<N, ROW_IN_F32>, g, kThreads, sm, st, a, nb);
        else launch_k(k_rows_r2c<N, ROW_IN_WEDGE>, g, kThreads, sm, st, a, nb);
    }
    static void rows_c2r(const RowC2RArgs& a, cudaStream_t st) {
        const int nb = (int)row_blocks();
        if constexpr (rows_lanes_ok<N>()) {
            if (lanes_form()) {
                const size_t sm = rows_lanes_smem_bytes<N>();
                static const int c = occ_ctas_t(k_rows_c2r_lanes<N>, kRowsLanesThreads, sm);
                launch_k(k_rows_c2r_lanes<N>, dim3((unsigned)c), kRowsLanesThreads, sm, st, a, a.nrows / 2);
                return;
            }
        }
        if constexpr (kRowsPl) {
            if (aligned16(a.src)) {
                static const int c = occ_ctas(k_rows_c2r_pl<N>, rows_c2r_pl_smem_bytes<N>());
                launch_k(k_rows_c2r_pl<N>, dim3((unsigned)(nb < c ? nb : c)), kThreads, rows_c2r_pl_smem_bytes<N>(), st,
                         a, nb);
                return;
            }
        }
        launch_k(k_rows_c2r<N>, (unsigned)(nb < pp_ctas() ? nb : pp_ctas()), kThreads, rows_smem_bytes<N>(), st, a, nb);
    }
    static void cols(const ColArgs& a, cudaStream_t st) {
        const dim3 g((unsigned)(col_tiles() - a.tile0));
        const size_t sm = cols_smem_bytes<N>();
        constexpr int kThreads = col_threads_of(N);
        const int ntiles = col_tiles() - a.tile0;
        if (a.dir < 0) {
            if (a.out_mode == COL_OUT_PLAIN) cols_plain<-1, COL_OUT_PLAIN>(a, ntiles, st);
            else if (a.out_mode == COL_OUT_BF16) cols_plain<-1, COL_OUT_BF16>(a, ntiles, st);
            else if (a.out_mode == COL_OUT_RING_F32) cols_plain<-1, COL_OUT_RING_F32>(a, ntiles, st);
            else cols_plain<-1, COL_OUT_WEDGE>(a, ntiles, st);
        } else {
            if (a.in_mode == COL_IN_PLAIN) cols_plain<1, COL_OUT_PLAIN>(a, ntiles, st);
            else if (a.in_mode == COL_IN_MAC_F32) launch_k(k_cols<N, 1, COL_IN_MAC_F32, COL_OUT_PLAIN>, g, kThreads, sm, st, a);
            else if (a.in_mode == COL_IN_MAC_BF16) launch_k(k_cols<N, 1, COL_IN_MAC_BF16, COL_OUT_PLAIN>, g, kThreads, sm, st, a);
            else if constexpr (!kColsPl) {
                // with the forward x pass of the newest slice (grids whose
                // plain x pass is k_cols_pp, whose arithmetic it repeats)
                if (a.in_mode == COL_IN_MAC_F32_X) launch_k(k_cols<N, 1, COL_IN_MAC_F32_X, COL_OUT_PLAIN>, g, kThreads, sm, st, a);
                else launch_k(k_cols<N, 1, COL_IN_MAC_BF16_X, COL_OUT_PLAIN>, g, kThreads, sm, st, a);
            }
        }
    }
};

} // namespace lc
