// lc_mac.cuh -- the shell multiply-accumulate (Eq. 13 summed over the active
// slices, steps 5-6 of Section 2.2) fused with the inverse x pass, for the
// full 16-column tiles of the half spectrum:
//
//   Jhat(p, q, r) = sum_j  Ghat_j(w(p, q, r)) * D_j * fhat_{s-j}(p, q, r)
//
// One CTA owns the tile (all p, line q, columns r in [c*CW, c*CW + CW)).
//  * ring tiles: the ring is [tile][slot][elements], so the tile's history
//    over all slots is one contiguous run; a slice's tile is one block of it,
//    brought in by one bulk asynchronous copy (cp.async.bulk, completion on
//    an mbarrier) per slice in an S-stage pipeline issued by thread 0; every
//    wait is bounded and reports a timeout in the plan's error word instead
//    of spinning;
//  * Ghat: the table is [wedge][A_pad] (slices of a wedge point contiguous);
//    the tile needs the rows w(p', q, r) for p' = min(p, N - p), so blocks of
//    8 slices are staged through shared memory, one 32-byte sector per
//    distinct row, shared by p and N - p;
//  * the sum stays in registers, then goes through the shared-memory x
//    transform and out to the work spectrum.
// The k = 0 mode is replaced by its FP64 value.
#pragma once
#include "lc_kernels.cuh"

namespace lc {

struct MacArgs {
    const void* ring;      // [tile][slot][tile elements]
    long long slot_elems;  // complex elements per slot
    int step, A, gstride, n_ring;
    const int* slot_step;
    const double* slot_S;
    const long long* slot_total;
    const float* ghat; // [W][gstride]
    const double* g0;  // [A]
    float2* dst;       // work spectrum
    const float2* tw;
    int* err;          // bit 4: a pipeline wait gave up
    int bf16;
    int instant;       // 1: every shell uses the observing step's slice (Eq. 18)
};

constexpr int kGBlock = 8;     // slices per staged Ghat block
constexpr int kGRow = kGBlock + 1; // padded smem row (bank-conflict free)

template <int N, bool BF16> struct MacCfg {
    static constexpr int CW = cw_of(N), NRP = nrp_of(N), M = N / 2, NCH = M / CW, BP = odd_pad(CW);
    static constexpr int NT = col_threads_of(N), NWARPS = NT / 32;
    static constexpr int TILE = N * CW, PER = (TILE + NT - 1) / NT;
    static constexpr int EB = BF16 ? 4 : 8;                  // bytes per ring element
    static constexpr int STAGE_BYTES = TILE * EB;
    static constexpr int GROWS = (M + 1) * CW;              // distinct Ghat rows of a tile
    static constexpr int GLOADS = (2 * GROWS + NT - 1) / NT; // float4 Ghat loads per thread per block
    static constexpr size_t G_BYTES = ((size_t)GROWS * kGRow * 4 + 127) / 128 * 128;
    static constexpr size_t FIXED = G_BYTES + (size_t)N * 8 + (size_t)kMaxShells * 12 + 2 * 8 * 8 + 256;
    static constexpr size_t BUDGET = 227 * 1024;
    // as many stages (<= 8) as the shared memory holds; the x-transform
    // buffer reuses the stage area once the MAC loop is done
    static constexpr int FIT = BUDGET > FIXED ? (int)((BUDGET - FIXED) / STAGE_BYTES) : 0;
    static constexpr int STAGES = FIT > 8 ? 8 : FIT;
    static constexpr size_t STAGE_AREA = (size_t)STAGES * STAGE_BYTES > (size_t)N * BP * 8
                                             ? (size_t)STAGES * STAGE_BYTES : (size_t)N * BP * 8;
    // shared memory layout (bytes)
    static constexpr size_t OFF_STAGE = 0;                                     // 128-B aligned
    static constexpr size_t OFF_G = (OFF_STAGE + STAGE_AREA + 127) / 128 * 128;
    static constexpr size_t OFF_TW = OFF_G + G_BYTES;
    static constexpr size_t OFF_LIST = OFF_TW + (size_t)N * 8;
    static constexpr size_t OFF_BAR = (OFF_LIST + (size_t)kMaxShells * 12 + 15) / 16 * 16;
    static constexpr size_t SMEM = OFF_BAR + 2 * 8 * 8 + 128; // full + empty barriers, alignment slack
    // the fused bulk-copy MAC serves grids whose tiles are 16 columns wide,
    // with at least 2 pipeline stages in shared memory
    static constexpr bool OK = N >= 32 && N <= 256 && STAGES >= 2 && SMEM <= BUDGET;
};

template <int N, bool BF16>
__global__ void __launch_bounds__(MacCfg<N, BF16>::NT) k_mac_tma(MacArgs a) {
    using C = MacCfg<N, BF16>;
    constexpr int NT = C::NT, CW = C::CW, PER = C::PER, TILE = C::TILE, BP = C::BP, S = C::STAGES;
    extern __shared__ unsigned char smem_raw2[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw2) + 127) & ~uintptr_t(127));
    unsigned char* stage = sm + C::OFF_STAGE;
    float2* buf = reinterpret_cast<float2*>(sm + C::OFF_STAGE); // after the MAC loop only
    float* gblk = reinterpret_cast<float*>(sm + C::OFF_G);
    float2* tw = reinterpret_cast<float2*>(sm + C::OFF_TW);
    int* s_slot = reinterpret_cast<int*>(sm + C::OFF_LIST);
    int* s_j = s_slot + kMaxShells;
    float* s_D = reinterpret_cast<float*>(s_j + kMaxShells);
    unsigned long long* full = reinterpret_cast<unsigned long long*>(sm + C::OFF_BAR);
    unsigned long long* empty = full + 8;
    __shared__ int s_nv, s_fail;
    __shared__ double s_dc;

    const int tile = blockIdx.x; // full tiles only
    const int line = tile / C::NCH, chunk = tile % C::NCH;
    const bool dc_tile = line == 0 && chunk == 0;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x < 32)
        mac_slot_list(a.A, a.step, a.n_ring, a.slot_step, a.slot_total, a.slot_S, a.g0, a.bf16 != 0, s_slot, s_j, s_D,
                      &s_nv, &s_dc, a.instant);
    if (threadIdx.x == 0) {
        s_fail = 0;
        for (int s = 0; s < S; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), C::NWARPS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = threadIdx.x; i < N; i += NT) tw[i] = a.tw[i];
    __syncthreads();
    const int nv = s_nv;
    // this tile's run of n_ring blocks
    const unsigned char* ring_tile =
        static_cast<const unsigned char*>(a.ring) + (size_t)tile * a.n_ring * C::STAGE_BYTES;
    auto issue = [&](int v) {
        const int st = v % S;
        const unsigned bar = smem_u32(&full[st]);
        mbar_expect_tx(bar, C::STAGE_BYTES);
        bulk_load(smem_u32(stage + (size_t)st * C::STAGE_BYTES), ring_tile + (size_t)s_slot[v] * C::STAGE_BYTES,
                  C::STAGE_BYTES, bar);
    };
    if (threadIdx.x == 0)
        for (int v = 0; v < nv && v < S; ++v) issue(v);

    // Ghat rows of the tile: row = p' * CW + col, wedge w(p', q, r)
    long long gbase[C::GLOADS];
#pragma unroll
    for (int k = 0; k < C::GLOADS; ++k) {
        const int rr = threadIdx.x + k * NT;
        const int row = rr >> 1, half = rr & 1;
        gbase[k] = rr < 2 * C::GROWS
                       ? wedge_of(row / CW, line, chunk * CW + row % CW, N) * a.gstride + half * 4
                       : -1;
    }
    float4 gpre[C::GLOADS];
    auto gfetch = [&](int blk) {
#pragma unroll
        for (int k = 0; k < C::GLOADS; ++k)
            if (gbase[k] >= 0) gpre[k] = __ldg(reinterpret_cast<const float4*>(a.ghat + gbase[k] + blk * kGBlock));
    };
    auto gstore = [&]() {
#pragma unroll
        for (int k = 0; k < C::GLOADS; ++k) {
            const int rr = threadIdx.x + k * NT;
            if (gbase[k] >= 0) {
                float* d = gblk + (rr >> 1) * kGRow + (rr & 1) * 4;
                d[0] = gpre[k].x;
                d[1] = gpre[k].y;
                d[2] = gpre[k].z;
                d[3] = gpre[k].w;
            }
        }
    };

    // this thread's elements: tile index idx -> (t = p, col)
    int grow[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int idx = threadIdx.x + i * NT;
        const int t = idx / CW, col = idx % CW;
        const int pf = t <= N - t ? t : N - t;
        grow[i] = (pf * CW + col) * kGRow;
    }
    float2 acc[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) acc[i] = make_float2(0.f, 0.f);

    int cur_blk = -1, pre_blk = -1;
    if (nv > 0) {
        pre_blk = s_j[0] / kGBlock;
        gfetch(pre_blk);
    }
    bool ok = true;
    for (int v = 0; v < nv; ++v) {
        const int j = s_j[v];
        const int blk = j / kGBlock;
        if (blk != cur_blk) {
            // switch the staged Ghat block (slices [8 blk, 8 blk + 8)); the next
            // block's rows are fetched into registers while this one is used
            __syncthreads();
            if (pre_blk != blk) gfetch(blk);
            gstore();
            __syncthreads();
            cur_blk = blk;
            pre_blk = blk + 1;
            if ((blk + 1) * kGBlock < a.A) gfetch(blk + 1);
        }
        const int st = v % S;
        const unsigned par = (unsigned)((v / S) & 1);
        ok = mbar_wait_bounded(smem_u32(&full[st]), par) && ok;
        const int jj = j - blk * kGBlock;
        const float D = s_D[v];
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int idx = threadIdx.x + i * NT;
            if (TILE % NT == 0 || idx < TILE) {
                float2 f;
                if constexpr (BF16) {
                    const __nv_bfloat162 h =
                        reinterpret_cast<const __nv_bfloat162*>(stage + (size_t)st * C::STAGE_BYTES)[idx];
                    f = __bfloat1622float2(h);
                } else {
                    f = reinterpret_cast<const float2*>(stage + (size_t)st * C::STAGE_BYTES)[idx];
                }
                const float g = gblk[grow[i] + jj] * D;
                acc[i].x = fmaf(g, f.x, acc[i].x);
                acc[i].y = fmaf(g, f.y, acc[i].y);
            }
        }
        // release the stage: one arrival per warp; the producer refills it
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&empty[st]));
        if (threadIdx.x == 0 && v + S < nv) {
            ok = mbar_wait_bounded(smem_u32(&empty[st]), par) && ok;
            issue(v + S);
        }
    }
    if (!ok) {
        atomicOr(&s_fail, 1);
        // give copies still in flight a second bounded wait before the CTA
        // (and its shared memory) goes away
        for (int v = nv - S > 0 ? nv - S : 0; v < nv; ++v)
            mbar_wait_bounded(smem_u32(&full[v % S]), (unsigned)((v / S) & 1));
    }
    __syncthreads(); // every stage consumed: the stage area becomes the x-transform buffer
    if (s_fail && threadIdx.x == 0) atomicOr(a.err, 4);
    if (dc_tile && threadIdx.x == 0) acc[0] = make_float2((float)s_dc, 0.0f);
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int idx = threadIdx.x + i * NT;
        if (TILE % NT == 0 || idx < TILE) buf[(idx / CW) * BP + (idx % CW)] = acc[i];
    }
    __syncthreads();
    fft_smem<N, 1, CW, BP, NT>(buf, tw);
    constexpr long long PLANE = (long long)N * C::NRP;
    const long long base = (long long)line * C::NRP + chunk * CW;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int idx = threadIdx.x + i * NT;
        if (TILE % NT == 0 || idx < TILE) {
            const int t = idx / CW, col = idx % CW;
            a.dst[base + t * PLANE + col] = buf[t * BP + col];
        }
    }
}

// ---------------------------------------------------------------------------
// Warp-specialised form of the same MAC (k_mac_ws).  The CTA has NC consumer
// threads and two producer warps:
//  * the ring producer streams the slices of the CTA's tiles through an
//    S-stage ring of shared-memory buffers (cp.async.bulk, lane 0);
//  * the Ghat producer gathers the Ghat rows those tiles share, in blocks of
//    4 slices (one 16-byte cp.async per row, all lanes, completion counted on
//    an mbarrier), double buffered, independently of the ring's progress;
//  * a consumer thread owns UPT units; a unit is a row pair {p, N - p}
//    (or {0, N/2}) times 4 consecutive columns, whose elements share the
//    Ghat values of wedge rows (min(p, N - p), q, r..r+3); the ring data is
//    read with 128-bit shared loads;
//  * consumers only wait for data and release buffers; the producers alone
//    wait for free buffers.  Every wait is bounded.
// PAIR = true: a CTA takes the tiles of lines q and N - q (same chunk),
// whose Ghat rows are the same, so each gathered row serves both and the
// gather traffic per ring byte halves; lines 0 and N/2 and the Nyquist tiles
// (CW lines q of the column r = N/2) go one per CTA.  PAIR = false: one tile
// per CTA.  Either way the launch covers every tile of the half spectrum.
// Arithmetic per element and slice is that of k_mac_tma and of the gather
// pass (g = Ghat * D, then two fused multiply-adds) in the same slice order,
// so all of them give identical sums.
constexpr int kWsGB = 4; // slices per Ghat block (16 bytes of a wedge row)

template <int N, bool BF16, bool PAIR> struct MacWsCfg {
    static constexpr int CW = cw_of(N), NRP = nrp_of(N), M = N / 2, NCH = M / CW, BP = odd_pad(CW);
    static constexpr int P = PAIR ? 2 : 1;            // tiles per CTA
    static constexpr int BPP = odd_pad(P * CW);       // x-transform buffer row (both tiles side by side)
    static constexpr int TILE = N * CW;
    static constexpr int EB = BF16 ? 4 : 8;
    static constexpr int TILE_BYTES = TILE * EB;      // one slice of one tile
    static constexpr int STAGE_BYTES = P * TILE_BYTES;
    static constexpr int CG = CW / 4;                 // 4-column groups
    static constexpr int UNITS = M * CG;              // (row pair, column group)
    static constexpr int UPT = PAIR && BF16 ? 1 : 2;  // units per consumer thread
    static constexpr int NC = UNITS / UPT;            // consumer threads
    static constexpr int NCW = NC / 32;               // consumer warps
    static constexpr int GW = BF16 && PAIR ? 3 : 2;   // Ghat producer warps
    static constexpr int NT = NC + 32 + 32 * GW;      // + the ring and the Ghat producer warps
    static constexpr int GROWS = (M + 1) * CW;        // distinct Ghat rows of a tile
    static constexpr int GPLANE = (M + 1) * CG;       // Ghat rows per column residue (col mod 4)
    static constexpr int GBLK_BYTES = GROWS * 16;     // one Ghat block: 4 floats per row
    static constexpr int MAXBLK = kMaxShells / kWsGB;
    static constexpr int GRID = PAIR ? (M + 1) * NCH + N / CW : N * NCH + N / CW;
    static constexpr size_t FIXED = 2 * (size_t)GBLK_BYTES + (size_t)GROWS * 4 + (size_t)N * 8 +
                                    (size_t)kMaxShells * 12 + (size_t)MAXBLK * 12 + 64 + 256;
    static constexpr size_t BUDGET = 227 * 1024;
    static constexpr int FIT = BUDGET > FIXED ? (int)((BUDGET - FIXED) / STAGE_BYTES) : 0;
    static constexpr int STAGES = FIT > 8 ? 8 : FIT;
    static constexpr size_t STAGE_AREA = (size_t)STAGES * STAGE_BYTES > (size_t)N * BPP * 8
                                             ? (size_t)STAGES * STAGE_BYTES : (size_t)N * BPP * 8;
    static constexpr size_t OFF_STAGE = 0;
    static constexpr size_t OFF_G = (OFF_STAGE + STAGE_AREA + 127) / 128 * 128;
    static constexpr size_t OFF_WROW = OFF_G + 2 * (size_t)GBLK_BYTES;
    static constexpr size_t OFF_TW = (OFF_WROW + (size_t)GROWS * 4 + 15) / 16 * 16;
    static constexpr size_t OFF_LIST = OFF_TW + (size_t)N * 8;
    static constexpr size_t OFF_BLK = OFF_LIST + (size_t)kMaxShells * 12;
    static constexpr size_t OFF_BAR = (OFF_BLK + (size_t)MAXBLK * 12 + 15) / 16 * 16;
    static constexpr int NBAR = 2 * 8 + 4; // full[8], empty[8], gfull[2], gempty[2]
    static constexpr size_t SMEM = OFF_BAR + NBAR * 8 + 128;
    // built where a tile has 4096 elements at most (16 columns up to N = 256,
    // 8 above) and the ring holds at least 2 stages (3 when a stage carries
    // two tiles)
    static constexpr bool OK = N >= 32 && N <= 512 && CW % 4 == 0 && TILE <= 4096 &&
                               STAGES >= (PAIR ? 3 : 2) && NC % 32 == 0 && UNITS % UPT == 0 && SMEM <= BUDGET;
};

__device__ __forceinline__ void cp_async16(unsigned dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(reinterpret_cast<unsigned long long>(src))
                 : "memory");
}
// arrive on the mbarrier once every cp.async issued so far by this thread has landed
__device__ __forceinline__ void cp_async_mbar_arrive(unsigned bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
// complex from a BF16 pair (low half: real part)
__device__ __forceinline__ float2 bf2_to_f2(unsigned w) {
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}

// mac_slot_list over the whole CTA: warp w takes rounds of 32 slices w,
// w + NW, ..., all of whose metadata loads are issued at once, instead of
// one warp walking the rounds.  The compaction keeps increasing lookback j,
// and the FP64 k = 0 sum adds the same per-round partials (lane 0 of each
// round's shuffle tree) in the same round order, so the list and the sum are
// identical to mac_slot_list's.  Every thread of the CTA calls it.
template <int NW>
__device__ __forceinline__ void ws_slot_list(const MacArgs& a, int* out_slot, int* out_j, float* out_D, int* nv_out,
                                             double* dc_out, int* s_wcnt, double* s_wdc) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int nv = 0;      // thread 0's running count and sum
    double dc = 0.0;
    for (int r0 = 0; r0 * 32 < a.A; r0 += NW) {
        const int round = r0 + warp;
        const int j = round * 32 + lane;
        const int n = a.instant ? a.step : a.step - j;
        bool valid = false;
        int slot = 0;
        double lum = 0.0, part = 0.0;
        if (j < a.A && n >= 0) {
            slot = n % a.n_ring;
            const int ss = a.slot_step[slot];
            const long long tot = a.slot_total[slot];
            const double S = a.slot_S[slot];
            const double g = a.g0[j];
            if (ss == n && tot != 0) {
                valid = true;
                lum = S * (double)tot;
                part = g * lum;
            }
        }
        const unsigned ball = __ballot_sync(0xffffffffu, valid);
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if (lane == 0) {
            s_wcnt[warp] = round * 32 < a.A ? __popc(ball) : 0;
            s_wdc[warp] = part;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            // rounds in order: exclusive prefix of the counts, and the k = 0 sum
            for (int w = 0; w < NW && (r0 + w) * 32 < a.A; ++w) {
                const int c = s_wcnt[w];
                s_wcnt[w] = nv;
                nv += c;
                dc += s_wdc[w];
            }
        }
        __syncthreads();
        if (valid) {
            const int pos = s_wcnt[warp] + __popc(ball & ((1u << lane) - 1u));
            out_slot[pos] = slot;
            out_j[pos] = j;
            out_D[pos] = a.bf16 ? (float)lum : 1.0f;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *nv_out = nv;
        *dc_out = dc;
    }
}

template <int N, bool BF16, bool PAIR>
__global__ void __launch_bounds__(MacWsCfg<N, BF16, PAIR>::NT, 1) k_mac_ws(MacArgs a) {
    using C = MacWsCfg<N, BF16, PAIR>;
    constexpr int NT = C::NT, NC = C::NC, CW = C::CW, TILE = C::TILE, BPP = C::BPP, S = C::STAGES, M = C::M;
    constexpr int UPT = C::UPT, CG = C::CG, GROWS = C::GROWS, GPLANE = C::GPLANE, P = C::P, NCH = C::NCH;
    extern __shared__ unsigned char smem_raw3[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw3) + 127) & ~uintptr_t(127));
    unsigned char* stage = sm + C::OFF_STAGE;
    float2* buf = reinterpret_cast<float2*>(sm + C::OFF_STAGE); // after the MAC loop only
    unsigned char* gsm = sm + C::OFF_G;
    int* s_wrow = reinterpret_cast<int*>(sm + C::OFF_WROW);
    float2* tw = reinterpret_cast<float2*>(sm + C::OFF_TW);
    int* s_slot = reinterpret_cast<int*>(sm + C::OFF_LIST);
    int* s_j = s_slot + kMaxShells;
    float* s_D = reinterpret_cast<float*>(s_j + kMaxShells);
    int* s_blk = reinterpret_cast<int*>(sm + C::OFF_BLK); // Ghat block of each block in use
    int* s_bmask = s_blk + C::MAXBLK;                     // its valid slices (bit jj)
    int* s_bv0 = s_bmask + C::MAXBLK;                     // index of its first valid slice
    unsigned long long* full = reinterpret_cast<unsigned long long*>(sm + C::OFF_BAR);
    unsigned long long* empty = full + 8;
    unsigned long long* gfull = full + 16;
    unsigned long long* gempty = full + 18;
    __shared__ int s_nv, s_nb, s_fail;
    __shared__ double s_dc;
    __shared__ int s_wcnt[NT / 32];
    __shared__ double s_wdc[NT / 32];

    // the CTA's tiles.  A full tile is (line q, columns [chunk CW, chunk CW + CW)),
    // a Nyquist tile (lines [line, line + CW), column N/2); element (t, col) of
    // tile h goes to dst[base[h] + t * N * NRP + col * cs]
    int tile[2], line, chunk = 0;
    bool nyq = false, two = false;
    long long base[2], cs = 1;
    {
        const int b = blockIdx.x;
        if (PAIR && b < (M - 1) * NCH) {
            line = 1 + b / NCH;
            chunk = b % NCH;
            two = true;
        } else if (PAIR && b < (M + 1) * NCH) {
            const int k = b - (M - 1) * NCH;
            line = k < NCH ? 0 : M;
            chunk = k % NCH;
        } else {
            const int t0 = PAIR ? b - (M + 1) * NCH + N * NCH : b;
            nyq = t0 >= N * NCH;
            line = nyq ? (t0 - N * NCH) * CW : t0 / NCH;
            chunk = nyq ? 0 : t0 % NCH;
        }
        if (nyq) {
            tile[0] = N * NCH + line / CW;
            base[0] = (long long)line * C::NRP + M;
            cs = C::NRP;
        } else {
            tile[0] = line * NCH + chunk;
            base[0] = (long long)line * C::NRP + chunk * CW;
        }
        tile[1] = two ? (N - line) * NCH + chunk : tile[0];
        base[1] = two ? (long long)(N - line) * C::NRP + chunk * CW : base[0];
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    ws_slot_list<NT / 32>(a, s_slot, s_j, s_D, &s_nv, &s_dc, s_wcnt, s_wdc);
    if (threadIdx.x == 32) {
        s_fail = 0;
        for (int i = 0; i < S; ++i) {
            mbar_init(smem_u32(&full[i]), 1);
            mbar_init(smem_u32(&empty[i]), C::NCW);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(&gfull[i]), 32 * C::GW);
            mbar_init(smem_u32(&gempty[i]), C::NCW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = threadIdx.x; i < N; i += NT) tw[i] = a.tw[i];
    // wedge rows of the tile(s), row = p' * CW + col (lines q and N - q share them)
    for (int r = threadIdx.x; r < GROWS; r += NT) {
        const int col = r % CW;
        s_wrow[r] = nyq ? (int)wedge_of(r / CW, line + col, M, N) : (int)wedge_of(r / CW, line, chunk * CW + col, N);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        // the Ghat blocks in slice order, with their valid slices: a block
        // starts at every v whose block differs from v - 1's, and its lane
        // collects the (at most kWsGB) slices that follow in it
        const int lane = threadIdx.x;
        int nb = 0;
        for (int v0 = 0; v0 < s_nv; v0 += 32) {
            const int v = v0 + lane;
            int b = 0;
            bool start = false;
            if (v < s_nv) {
                b = s_j[v] / kWsGB;
                start = v == 0 || s_j[v - 1] / kWsGB != b;
            }
            const unsigned ball = __ballot_sync(0xffffffffu, start);
            if (start) {
                const int pos = nb + __popc(ball & ((1u << lane) - 1u));
                int mask = 0;
                for (int k = v; k < s_nv && s_j[k] / kWsGB == b; ++k) mask |= 1 << (s_j[k] - b * kWsGB);
                s_blk[pos] = b;
                s_bmask[pos] = mask;
                s_bv0[pos] = v;
            }
            nb += __popc(ball);
        }
        if (lane == 0) s_nb = nb;
    }
    __syncthreads();
    const int nv = s_nv, nb = s_nb;
    bool ok = true;
    // consumer state: unit u = threadIdx.x + k * NC is row pair pu = u / CG,
    // columns 4 cg .. 4 cg + 3, in each of the CTA's tiles h
    float2 accA[P][UPT][4], accB[P][UPT][4];
#pragma unroll
    for (int h = 0; h < P; ++h)
#pragma unroll
        for (int k = 0; k < UPT; ++k)
#pragma unroll
            for (int c = 0; c < 4; ++c) accA[h][k][c] = accB[h][k][c] = make_float2(0.f, 0.f);

    if (warp == C::NCW) {
        // ------------------------------------------------------- ring producer
        const unsigned char* ring0 = static_cast<const unsigned char*>(a.ring) + (size_t)tile[0] * a.n_ring * C::TILE_BYTES;
        const unsigned char* ring1 = static_cast<const unsigned char*>(a.ring) + (size_t)tile[1] * a.n_ring * C::TILE_BYTES;
        if (lane == 0) {
            for (int v = 0; v < nv; ++v) {
                const int st = v % S;
                if (v >= S) ok = mbar_wait_bounded(smem_u32(&empty[st]), (unsigned)(((v / S) - 1) & 1)) && ok;
                const unsigned bar = smem_u32(&full[st]);
                unsigned char* dst0 = stage + (size_t)st * C::STAGE_BYTES;
                mbar_expect_tx(bar, two ? 2 * C::TILE_BYTES : C::TILE_BYTES);
                bulk_load(smem_u32(dst0), ring0 + (size_t)s_slot[v] * C::TILE_BYTES, C::TILE_BYTES, bar);
                if (two)
                    bulk_load(smem_u32(dst0 + C::TILE_BYTES), ring1 + (size_t)s_slot[v] * C::TILE_BYTES, C::TILE_BYTES,
                              bar);
            }
        }
        __syncwarp();
    } else if (warp > C::NCW) {
        // ------------------------------------------------------ Ghat producers
        // (run up to two blocks ahead of the consumers, whatever the ring does;
        // GW warps share the rows of a block)
        const int gl = lane + 32 * (warp - C::NCW - 1);
        for (int gi = 0; gi < nb; ++gi) {
            const int gb = gi & 1;
            if (gi >= 2) ok = mbar_wait_bounded(smem_u32(&gempty[gb]), (unsigned)(((gi >> 1) - 1) & 1)) && ok;
            // Ghat rows of block s_blk[gi]: row (p', col) goes to slot (col % 4) * GPLANE + p' * CG + col / 4
            const float* gsrc = a.ghat + (size_t)s_blk[gi] * kWsGB;
            const unsigned gdst = smem_u32(gsm + (size_t)gb * C::GBLK_BYTES);
            for (int r = gl; r < GROWS; r += 32 * C::GW) {
                const int pp = r / CW, col = r % CW;
                cp_async16(gdst + ((col & 3) * GPLANE + pp * CG + (col >> 2)) * 16,
                           gsrc + (size_t)s_wrow[r] * a.gstride);
            }
            cp_async_mbar_arrive(smem_u32(&gfull[gb]));
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else {
        // ------------------------------------------------------------ consumers
        int offA[UPT], offB[UPT], goffA[UPT], goffB[UPT];
#pragma unroll
        for (int k = 0; k < UPT; ++k) {
            const int u = threadIdx.x + k * NC;
            const int pu = u / CG, cg = u % CG;
            offA[k] = (pu * CW + cg * 4) * C::EB;                    // byte offset in a tile's slice
            offB[k] = ((pu == 0 ? M : N - pu) * CW + cg * 4) * C::EB;
            goffA[k] = (pu * CG + cg) * 16;                          // Ghat slot of column residue 0
            goffB[k] = ((pu == 0 ? M : pu) * CG + cg) * 16;
        }
        for (int gi = 0; gi < nb; ++gi) {
            const int gb = gi & 1;
            ok = mbar_wait_bounded(smem_u32(&gfull[gb]), (unsigned)((gi >> 1) & 1)) && ok;
            const unsigned char* gblk = gsm + (size_t)gb * C::GBLK_BYTES;
            float4 gA[UPT][4], gB[UPT][4];
#pragma unroll
            for (int k = 0; k < UPT; ++k)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    gA[k][c] = *reinterpret_cast<const float4*>(gblk + c * GPLANE * 16 + goffA[k]);
                    gB[k][c] = *reinterpret_cast<const float4*>(gblk + c * GPLANE * 16 + goffB[k]);
                }
            const int mask = s_bmask[gi];
            int v = s_bv0[gi];
#pragma unroll
            for (int jj = 0; jj < kWsGB; ++jj) {
                if (!(mask & (1 << jj))) continue;
                const int st = v % S;
                ok = mbar_wait_bounded(smem_u32(&full[st]), (unsigned)((v / S) & 1)) && ok;
                const float D = s_D[v];
#pragma unroll
                for (int h = 0; h < P; ++h) {
                    if (h == 1 && !two) continue;
                    const unsigned char* sb = stage + (size_t)st * C::STAGE_BYTES + h * C::TILE_BYTES;
#pragma unroll
                    for (int k = 0; k < UPT; ++k) {
                        float2 fA[4], fB[4];
                        if constexpr (BF16) {
                            const uint4 wa = *reinterpret_cast<const uint4*>(sb + offA[k]);
                            const uint4 wb = *reinterpret_cast<const uint4*>(sb + offB[k]);
                            fA[0] = bf2_to_f2(wa.x); fA[1] = bf2_to_f2(wa.y);
                            fA[2] = bf2_to_f2(wa.z); fA[3] = bf2_to_f2(wa.w);
                            fB[0] = bf2_to_f2(wb.x); fB[1] = bf2_to_f2(wb.y);
                            fB[2] = bf2_to_f2(wb.z); fB[3] = bf2_to_f2(wb.w);
                        } else {
                            const float4 a0 = *reinterpret_cast<const float4*>(sb + offA[k]);
                            const float4 a1 = *reinterpret_cast<const float4*>(sb + offA[k] + 16);
                            const float4 b0 = *reinterpret_cast<const float4*>(sb + offB[k]);
                            const float4 b1 = *reinterpret_cast<const float4*>(sb + offB[k] + 16);
                            fA[0] = make_float2(a0.x, a0.y); fA[1] = make_float2(a0.z, a0.w);
                            fA[2] = make_float2(a1.x, a1.y); fA[3] = make_float2(a1.z, a1.w);
                            fB[0] = make_float2(b0.x, b0.y); fB[1] = make_float2(b0.z, b0.w);
                            fB[2] = make_float2(b1.x, b1.y); fB[3] = make_float2(b1.z, b1.w);
                        }
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const float ga = jj == 0 ? gA[k][c].x : jj == 1 ? gA[k][c].y : jj == 2 ? gA[k][c].z : gA[k][c].w;
                            const float gbv = jj == 0 ? gB[k][c].x : jj == 1 ? gB[k][c].y : jj == 2 ? gB[k][c].z : gB[k][c].w;
                            const float g1 = ga * D, g2 = gbv * D;
                            accA[h][k][c].x = fmaf(g1, fA[c].x, accA[h][k][c].x);
                            accA[h][k][c].y = fmaf(g1, fA[c].y, accA[h][k][c].y);
                            accB[h][k][c].x = fmaf(g2, fB[c].x, accB[h][k][c].x);
                            accB[h][k][c].y = fmaf(g2, fB[c].y, accB[h][k][c].y);
                        }
                    }
                }
                // release the stage: one arrival per warp
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&empty[st]));
                ++v;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&gempty[gb]));
        }
        if (!ok) {
            atomicOr(&s_fail, 1);
            // give copies still in flight a second bounded wait before the
            // stage area is reused
            for (int v = nv - S > 0 ? nv - S : 0; v < nv; ++v)
                mbar_wait_bounded(smem_u32(&full[v % S]), (unsigned)((v / S) & 1));
        }
    }
    if (!ok) atomicOr(&s_fail, 1);
    __syncthreads(); // every stage consumed: the stage area becomes the x-transform buffer
    if (s_fail && threadIdx.x == 0) atomicOr(a.err, 4);
    if (warp < C::NCW) {
        if (!nyq && line == 0 && chunk == 0 && threadIdx.x == 0) accA[0][0][0] = make_float2((float)s_dc, 0.0f);
#pragma unroll
        for (int h = 0; h < P; ++h)
#pragma unroll
            for (int k = 0; k < UPT; ++k) {
                const int u = threadIdx.x + k * NC;
                const int pu = u / CG, cg = u % CG;
                const int tA = pu, tB = pu == 0 ? M : N - pu;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    buf[tA * BPP + h * CW + cg * 4 + c] = accA[h][k][c];
                    buf[tB * BPP + h * CW + cg * 4 + c] = accB[h][k][c];
                }
            }
    }
    __syncthreads();
    fft_smem<N, 1, P * CW, BPP, NT>(buf, tw);
    constexpr long long PLANE = (long long)N * C::NRP;
    for (int idx = threadIdx.x; idx < P * TILE; idx += NT) {
        const int h = idx / TILE, e = idx % TILE;
        if (h == 1 && !two) break;
        const int t = e / CW, col = e % CW;
        a.dst[base[h] + t * PLANE + col * cs] = buf[t * BPP + h * CW + col];
    }
}

template <int N, bool BF16, bool PAIR> struct MacWsLaunch {
    using C = MacWsCfg<N, BF16, PAIR>;
    static cudaError_t init() {
        if constexpr (!C::OK) return cudaSuccess;
        else return cudaFuncSetAttribute(k_mac_ws<N, BF16, PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    }
    // every tile of the half spectrum: full ones (paired or single), then the Nyquist ones
    static void run(const MacArgs& a, cudaStream_t st) {
        if constexpr (C::OK) launch_k(k_mac_ws<N, BF16, PAIR>, C::GRID, C::NT, C::SMEM, st, a);
    }
};

template <int N, bool BF16> struct MacLaunch {
    using C = MacCfg<N, BF16>;
    static cudaError_t init() {
        if constexpr (!C::OK) return cudaSuccess;
        else return cudaFuncSetAttribute(k_mac_tma<N, BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    }
    static void run(const MacArgs& a, cudaStream_t st) {
        if constexpr (C::OK) launch_k(k_mac_tma<N, BF16>, N * C::NCH, C::NT, C::SMEM, st, a);
    }
};

} // namespace lc
