// lc_mac.cuh -- the shell multiply-accumulate (Eq. 13 summed over the active
// slices, steps 5-6 of Section 2.2) fused with the inverse x pass, for the
// full 16-column tiles of the half spectrum:
//
//   Jhat(p, q, r) = sum_j  Ghat_j(w(p, q, r)) * D_j * fhat_{s-j}(p, q, r)
//
// One CTA owns the tile (all p, line q, columns r in [c*CW, c*CW + CW)).
//  * ring tiles: one TMA box per active slice (cp.async.bulk.tensor.4d over
//    the ring viewed as [slot][p][q][r]), an S-stage mbarrier pipeline issued
//    by thread 0; every wait is bounded and reports a timeout in the plan's
//    error word instead of spinning;
//  * Ghat: the table is [wedge][A_pad] (slices of a wedge point contiguous);
//    the tile needs the rows w(p', q, r) for p' = min(p, N - p), so blocks of
//    8 slices are staged through shared memory, one 32-byte sector per
//    distinct row, shared by p and N - p;
//  * the sum stays in registers, then goes through the shared-memory x
//    transform and out to the work spectrum.
// The k = 0 mode is replaced by its FP64 value.
#pragma once
#include <cuda.h>

#include "lc_kernels.cuh"

namespace lc {

struct MacArgs {
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
};

constexpr int kGBlock = 8;     // slices per staged Ghat block
constexpr int kGRow = kGBlock + 1; // padded smem row (bank-conflict free)

template <int N, bool BF16> struct MacCfg {
    static constexpr int CW = cw_of(N), NRP = nrp_of(N), M = N / 2, NCH = M / CW, BP = odd_pad(CW);
    // pipeline depth: 4 stages where the shared memory allows, else 2
    static constexpr int STAGES = (BF16 || N <= 128) ? 4 : 2;
    static constexpr int NT = col_threads_of(N);
    static constexpr int TILE = N * CW, PER = (TILE + NT - 1) / NT;
    static constexpr int EB = BF16 ? 4 : 8;                  // bytes per ring element
    static constexpr int STAGE_BYTES = TILE * EB;
    static constexpr int BOXES = N > 256 ? 2 : 1;           // TMA boxes per stage (p extent <= 256)
    static constexpr int GROWS = (M + 1) * CW;              // distinct Ghat rows of a tile
    // shared memory layout (bytes)
    static constexpr size_t OFF_STAGE = 0;                                     // 128-B aligned
    static constexpr size_t OFF_G = OFF_STAGE + (size_t)STAGES * STAGE_BYTES;
    static constexpr size_t OFF_BUF = (OFF_G + (size_t)GROWS * kGRow * 4 + 15) / 16 * 16;
    static constexpr size_t OFF_TW = OFF_BUF + (size_t)N * BP * 8;
    static constexpr size_t OFF_LIST = OFF_TW + (size_t)N * 8;
    static constexpr size_t OFF_BAR = (OFF_LIST + (size_t)kMaxShells * 12 + 15) / 16 * 16;
    static constexpr size_t SMEM = OFF_BAR + STAGES * 8 + 128; // + alignment slack
    // the fused TMA MAC serves grids whose tiles are 16 columns wide and whose
    // p extent fits one or two TMA boxes within the shared-memory budget
    static constexpr bool OK = N >= 32 && N <= 256 && SMEM <= 227 * 1024;
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
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
__device__ __forceinline__ void tma_load_4d(unsigned dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

template <int N, bool BF16>
__global__ void __launch_bounds__(MacCfg<N, BF16>::NT) k_mac_tma(const __grid_constant__ CUtensorMap ring, MacArgs a) {
    using C = MacCfg<N, BF16>;
    constexpr int NT = C::NT, CW = C::CW, PER = C::PER, TILE = C::TILE, M = C::M, BP = C::BP;
    extern __shared__ unsigned char smem_raw2[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw2) + 127) & ~uintptr_t(127));
    unsigned char* stage = sm + C::OFF_STAGE;
    float* gblk = reinterpret_cast<float*>(sm + C::OFF_G);
    float2* buf = reinterpret_cast<float2*>(sm + C::OFF_BUF);
    float2* tw = reinterpret_cast<float2*>(sm + C::OFF_TW);
    int* s_slot = reinterpret_cast<int*>(sm + C::OFF_LIST);
    int* s_j = s_slot + kMaxShells;
    float* s_D = reinterpret_cast<float*>(s_j + kMaxShells);
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(sm + C::OFF_BAR);
    __shared__ int s_nv, s_fail;
    __shared__ double s_dc;

    const int tile = blockIdx.x; // full tiles only
    const int line = tile / C::NCH, chunk = tile % C::NCH;
    const bool dc_tile = line == 0 && chunk == 0;

    if (threadIdx.x == 0) {
        int nv = 0;
        double dc = 0.0;
        for (int j = 0; j < a.A; ++j) {
            const int n = a.step - j;
            if (n < 0) break;
            const int slot = n % a.n_ring;
            if (a.slot_step[slot] != n) continue;
            const long long tot = a.slot_total[slot];
            if (tot == 0) continue;
            const double lum = a.slot_S[slot] * (double)tot;
            s_slot[nv] = slot;
            s_j[nv] = j;
            s_D[nv] = a.bf16 ? (float)lum : 1.0f;
            dc += a.g0[j] * lum;
            ++nv;
        }
        s_nv = nv;
        s_dc = dc;
        s_fail = 0;
        for (int s = 0; s < C::STAGES; ++s) mbar_init(smem_u32(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = threadIdx.x; i < N; i += NT) tw[i] = a.tw[i];
    __syncthreads();
    const int nv = s_nv;
    // ring coordinates: {r (elements), q, p, slot}; FP32 complex = 2 floats
    const int c0 = chunk * CW * (BF16 ? 1 : 2);
    auto issue = [&](int v) {
        const int st = v % C::STAGES;
        const unsigned bar = smem_u32(&bars[st]);
        mbar_expect_tx(bar, C::STAGE_BYTES);
#pragma unroll
        for (int b = 0; b < C::BOXES; ++b)
            tma_load_4d(smem_u32(stage + (size_t)st * C::STAGE_BYTES + (size_t)b * (C::STAGE_BYTES / C::BOXES)), &ring,
                        c0, line, b * (N / C::BOXES), s_slot[v], bar);
    };
    if (threadIdx.x == 0)
        for (int v = 0; v < nv && v < C::STAGES; ++v) issue(v);

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

    int cur_blk = -1;
    bool ok = true;
    for (int v = 0; v < nv; ++v) {
        const int j = s_j[v];
        const int blk = j / kGBlock;
        if (blk != cur_blk) {
            // stage Ghat rows w(p', q, r) for slices [8 blk, 8 blk + 8)
            __syncthreads();
            for (int rr = threadIdx.x; rr < C::GROWS * 2; rr += NT) {
                const int row = rr >> 1, half = rr & 1;
                const int pf = row / CW, col = row % CW;
                const float4 g4 = __ldg(reinterpret_cast<const float4*>(
                    a.ghat + wedge_of(pf, line, chunk * CW + col, N) * a.gstride + blk * kGBlock + half * 4));
                float* d = gblk + row * kGRow + half * 4;
                d[0] = g4.x;
                d[1] = g4.y;
                d[2] = g4.z;
                d[3] = g4.w;
            }
            __syncthreads();
            cur_blk = blk;
        }
        const int st = v % C::STAGES;
        ok = mbar_wait_bounded(smem_u32(&bars[st]), (unsigned)((v / C::STAGES) & 1)) && ok;
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
        __syncthreads(); // stage st consumed by every thread
        if (threadIdx.x == 0 && v + C::STAGES < nv) issue(v + C::STAGES);
    }
    if (!ok) {
        atomicOr(&s_fail, 1);
        // give copies still in flight a second bounded wait before the CTA
        // (and its shared memory) goes away
        for (int v = nv - C::STAGES > 0 ? nv - C::STAGES : 0; v < nv; ++v)
            mbar_wait_bounded(smem_u32(&bars[v % C::STAGES]), (unsigned)((v / C::STAGES) & 1));
    }
    __syncthreads();
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
    static void run(const CUtensorMap* map, const MacArgs& a, cudaStream_t st) {
        if constexpr (C::OK) k_mac_tma<N, BF16><<<N * C::NCH, C::NT, C::SMEM, st>>>(*map, a);
    }
};

} // namespace lc
