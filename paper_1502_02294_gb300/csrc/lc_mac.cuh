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

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
// bounded wait: ~2^22 polls with back-off (well over a second), then give up
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity) {
    for (int it = 0; it < (1 << 22); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it > 64) __nanosleep(128);
    }
    return false;
}
// one contiguous global -> shared copy, completion counted on an mbarrier
__device__ __forceinline__ void bulk_load(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(src)), "r"(bytes), "r"(bar)
        : "memory");
}

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

template <int N, bool BF16> struct MacLaunch {
    using C = MacCfg<N, BF16>;
    static cudaError_t init() {
        if constexpr (!C::OK) return cudaSuccess;
        else return cudaFuncSetAttribute(k_mac_tma<N, BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    }
    static void run(const MacArgs& a, cudaStream_t st) {
        if constexpr (C::OK) k_mac_tma<N, BF16><<<N * C::NCH, C::NT, C::SMEM, st>>>(a);
    }
};

} // namespace lc
