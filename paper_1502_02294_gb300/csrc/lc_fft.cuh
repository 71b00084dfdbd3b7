// lc_fft.cuh -- shared-memory mixed-radix FFT building blocks for sm_103a.
//
// The transforms of Eq. 12 (forward e^{-2 pi i k.x/N}, unnormalised; inverse
// e^{+2 pi i k.x/N}) are done as three axis passes over a half spectrum
// [p][q][r], r in [0, N/2], rows padded to NRP complex so that every row and
// every 16-column chunk starts on a 32-byte sector.
//
// One CTA holds B independent length-N transforms in shared memory as
// buf[t * BP + b] (transform b, element t; BP odd so that both the strided
// Stockham loads and the contiguous stores are bank-conflict free).  A
// radix-R stage loads every butterfly's R inputs into registers, waits,
// twiddles, applies the R-point DFT and stores in place (Stockham autosort:
// natural order in and out, no bit reversal).  Twiddles come from a table of
// W_N^m = e^{-2 pi i m / N}, computed in FP64 on the host.
#pragma once
#include <cuda.h> // CUtensorMap (the tensor maps of the TMA column passes)
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <utility>

namespace lc {

constexpr int kThreads = 256;

// Near field of the innermost shell: the displacements with |d|_inf <= kNearR
// are left out of the FFT path and added exactly in FP64 per source.
constexpr int kNearR = 2;
constexpr int kNearSide = 2 * kNearR + 1, kNearCube = kNearSide * kNearSide * kNearSide;
// wedge index of a near displacement (fold signs, sort)
__host__ __device__ __forceinline__ int near_wedge(int dx, int dy, int dz) {
    int a = dx < 0 ? -dx : dx, b = dy < 0 ? -dy : dy, c = dz < 0 ? -dz : dz, t;
    if (a > b) { t = a; a = b; b = t; }
    if (b > c) { t = b; b = c; c = t; }
    if (a > b) { t = a; a = b; b = t; }
    return c * (c + 1) * (c + 2) / 6 + b * (b + 1) / 2 + a;
}

// Near-field list of one push: per deposited source its cell and its integer
// share q; the innermost shell's near cube around each is summed exactly in
// FP64 into `acc` (one item per (source, cube cell), kNearCube per source).
struct NearScatter {
    const long long* cell;
    const long long* q;
    long long n;             // sources in the list
    const double* gnear;     // the innermost shell's near wedge (f_0 folded in)
    const double* slot_S;    // per-slot fixed-point unit
    int slot;
    double U;                // output unit
    double* acc;             // N^3 FP64 accumulator, zero where not yet folded
    int ctas;                // extra CTAs of a plane kernel that run the list (0: none)
};

// Item idx = s * kNearCube + m: source s, displacement m of its near cube
// (x slowest), target cell wrapped periodically on the N^3 grid.
__device__ __forceinline__ long long near_target(long long c, int m, int N, int& dx, int& dy, int& dz) {
    dx = m / (kNearSide * kNearSide) - kNearR;
    dy = (m / kNearSide) % kNearSide - kNearR;
    dz = m % kNearSide - kNearR;
    const long long NN = (long long)N * N;
    const int ix = (int)(c / NN), iy = (int)((c / N) % N), iz = (int)(c % N);
    const int tx = (ix + dx + N) % N, ty = (iy + dy + N) % N, tz = (iz + dz + N) % N;
    return ((long long)tx * N + ty) * N + tz;
}

__device__ __forceinline__ void near_scatter_item(const NearScatter& a, int N, long long idx) {
    const long long s = idx / kNearCube;
    const int m = (int)(idx % kNearCube);
    const long long qs = a.q[s];
    if (qs == 0) return;
    int dx, dy, dz;
    const long long t = near_target(a.cell[s], m, N, dx, dy, dz);
    atomicAdd(a.acc + t, a.U * a.slot_S[a.slot] * (double)qs * a.gnear[near_wedge(dx, dy, dz)]);
}

// Launch through cudaLaunchKernelEx (one launch path for every per-step
// kernel; no launch attributes).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                            Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = nullptr;
    cfg.numAttrs = 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// ---- thread-block clusters: rank, the peer's shared memory, barrier ----
__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// the shared::cluster address of `saddr` (a shared::cta address) in CTA `rank`
__device__ __forceinline__ unsigned cluster_map(unsigned saddr, unsigned rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
__device__ __forceinline__ void cluster_st(unsigned addr, float2 v) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ float2 cluster_ld(unsigned addr) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
    return v;
}
// every thread of every CTA of the cluster (no convergence assumed): the
// shared-memory writes before it, the peer's included, are visible to all
// after it
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// ---- asynchronous copies counted on shared-memory mbarriers ----
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

// one box of a tensor map (rank 3) -> shared memory, completion counted on
// an mbarrier; coordinates innermost first
__device__ __forceinline__ void tma_load_3d(unsigned dst, const void* tmap, int c0, int c1, int c2, unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(dst), "l"(reinterpret_cast<unsigned long long>(tmap)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}
// order this thread's earlier shared-memory accesses before later
// asynchronous-proxy (bulk copy) accesses of the same memory
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__host__ __device__ constexpr int nrp_of(int n) { return ((n / 2 + 1) + 7) / 8 * 8; }
// columns per x-pass tile: 16, or 8 from N = 384 up, so that a tile
// (N x CW elements) stays within 4096 elements and the shell MAC's pipeline
// fits in shared memory at every grid size
__host__ __device__ constexpr int cw_of(int n) { return n >= 384 ? 8 : (n / 2 < 16 ? n / 2 : 16); }
// pairs of real rows per CTA in the z (row) passes
__host__ __device__ constexpr int row_pairs_of(int n) {
    return n <= 8 ? 32 : n <= 16 ? 32 : n <= 32 ? 32 : n <= 64 ? 32 : n <= 128 ? 16 : n <= 256 ? 8 : 4;
}
__host__ __device__ constexpr int odd_pad(int b) { return (b % 2 == 0) ? b + 1 : b; }

// Radix plan: stages applied in order R0, R1, R2 (1 = unused).
template <int N> struct Plan;
template <> struct Plan<8> { static constexpr int R0 = 8, R1 = 1, R2 = 1; };
template <> struct Plan<16> { static constexpr int R0 = 16, R1 = 1, R2 = 1; };
template <> struct Plan<32> { static constexpr int R0 = 8, R1 = 4, R2 = 1; };
template <> struct Plan<64> { static constexpr int R0 = 8, R1 = 8, R2 = 1; };
template <> struct Plan<96> { static constexpr int R0 = 8, R1 = 4, R2 = 3; };
template <> struct Plan<128> { static constexpr int R0 = 16, R1 = 8, R2 = 1; };
template <> struct Plan<192> { static constexpr int R0 = 8, R1 = 8, R2 = 3; };
template <> struct Plan<256> { static constexpr int R0 = 16, R1 = 16, R2 = 1; };
template <> struct Plan<384> { static constexpr int R0 = 16, R1 = 8, R2 = 3; };
template <> struct Plan<512> { static constexpr int R0 = 8, R1 = 8, R2 = 8; };

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by DIR * i  (DIR = -1 forward, +1 inverse)
template <int DIR> __device__ __forceinline__ float2 mul_i(float2 a) {
    return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

// ---- small DFTs in registers: y_k = sum_n v_n e^{DIR 2 pi i n k / R} ----
template <int DIR> __device__ __forceinline__ void dft2(float2& a, float2& b) {
    float2 t = csub(a, b);
    a = cadd(a, b);
    b = t;
}

template <int DIR> __device__ __forceinline__ void dft3(float2* v) {
    const float h = 0.86602540378443864676f; // sqrt(3)/2
    float2 t = cadd(v[1], v[2]);
    float2 d = mul_i<DIR>(cscale(csub(v[1], v[2]), h));
    float2 m = make_float2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
    v[0] = cadd(v[0], t);
    v[1] = cadd(m, d);
    v[2] = csub(m, d);
}

// 4-point DFT on v[s*0], v[s*1], v[s*2], v[s*3]
template <int DIR, int S = 1> __device__ __forceinline__ void dft4(float2* v) {
    float2 t0 = cadd(v[0], v[2 * S]), t1 = csub(v[0], v[2 * S]);
    float2 t2 = cadd(v[S], v[3 * S]), t3 = mul_i<DIR>(csub(v[S], v[3 * S]));
    v[0] = cadd(t0, t2);
    v[2 * S] = csub(t0, t2);
    v[S] = cadd(t1, t3);
    v[3 * S] = csub(t1, t3);
}

template <int DIR> __device__ __forceinline__ void dft8(float2* v) {
    const float c = 0.70710678118654752440f;
    // even / odd halves
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    dft4<DIR>(e);
    dft4<DIR>(o);
    // W8^1 = c (1 + DIR i), W8^2 = DIR i, W8^3 = c (-1 + DIR i)
    float2 w1 = cscale(cadd(o[1], mul_i<DIR>(o[1])), c);
    float2 w2 = mul_i<DIR>(o[2]);
    float2 w3 = cscale(csub(mul_i<DIR>(o[3]), o[3]), c);
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], w1);
    v[5] = csub(e[1], w1);
    v[2] = cadd(e[2], w2);
    v[6] = csub(e[2], w2);
    v[3] = cadd(e[3], w3);
    v[7] = csub(e[3], w3);
}

// 16-point DFT as 4 x 4: n = 4a + b, k = k1 + 4 k2
template <int DIR> __device__ __forceinline__ void dft16(float2* v) {
    const float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f, c2 = 0.70710678118654752440f;
    // inner DFT4 over a for each b (stride 4 in v)
#pragma unroll
    for (int b = 0; b < 4; ++b) dft4<DIR, 4>(v + b);
    // now v[4*k1 + b] = X_b[k1]; twiddle by W16^{b k1} with W16 = e^{DIR 2 pi i / 16}
    const float ds = (float)DIR;
    // W16^m for m = 1..9 : (cos(2 pi m/16), DIR sin(2 pi m / 16))
    const float2 w1 = make_float2(c1, ds * s1), w2 = make_float2(c2, ds * c2), w3 = make_float2(s1, ds * c1);
    const float2 w6 = make_float2(-c2, ds * c2), w9 = make_float2(-c1, -ds * s1);
    v[4 * 1 + 1] = cmul(v[5], w1);
    v[4 * 1 + 2] = cmul(v[6], w2);
    v[4 * 1 + 3] = cmul(v[7], w3);
    v[4 * 2 + 1] = cmul(v[9], w2);
    v[4 * 2 + 2] = mul_i<DIR>(v[10]);
    v[4 * 2 + 3] = cmul(v[11], w6);
    v[4 * 3 + 1] = cmul(v[13], w3);
    v[4 * 3 + 2] = cmul(v[14], w6);
    v[4 * 3 + 3] = cmul(v[15], w9);
    // outer DFT4 over b for each k1 (contiguous groups of 4)
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<DIR, 1>(v + 4 * k1);
    // v[4 k1 + k2] = y[k1 + 4 k2]: transpose 4x4 into natural order
    float2 t[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) t[i] = v[i];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[4 * k1 + k2];
}

// 12-point DFT as 4 x 3: n = 3 a + b, k = k1 + 4 k2: a 4-point DFT over a for
// each b, the twiddle W12^(b k1), a 3-point DFT over b for each k1
template <int DIR> __device__ __forceinline__ void dft12(float2* v) {
    const float h = 0.86602540378443864676f; // sqrt(3)/2
    const float ds = (float)DIR;
    float2 a[3][4];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
#pragma unroll
        for (int q = 0; q < 4; ++q) a[b][q] = v[3 * q + b];
        dft4<DIR>(a[b]);
    }
    // W12^m = (cos(2 pi m / 12), DIR sin(2 pi m / 12)) for m = 1, 2, 3, 4, 6
    const float2 w1 = make_float2(h, ds * 0.5f), w2 = make_float2(0.5f, ds * h);
    const float2 w4 = make_float2(-0.5f, ds * h);
    a[1][1] = cmul(a[1][1], w1);
    a[1][2] = cmul(a[1][2], w2);
    a[1][3] = mul_i<DIR>(a[1][3]); // W12^3 = DIR i
    a[2][1] = cmul(a[2][1], w2);
    a[2][2] = cmul(a[2][2], w4);
    a[2][3] = make_float2(-a[2][3].x, -a[2][3].y); // W12^6 = -1
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        float2 t[3] = {a[0][k1], a[1][k1], a[2][k1]};
        dft3<DIR>(t);
#pragma unroll
        for (int k2 = 0; k2 < 3; ++k2) v[k1 + 4 * k2] = t[k2];
    }
}

template <int R, int DIR> __device__ __forceinline__ void dft(float2* v) {
    if constexpr (R == 2) dft2<DIR>(v[0], v[1]);
    else if constexpr (R == 3) dft3<DIR>(v);
    else if constexpr (R == 4) dft4<DIR>(v);
    else if constexpr (R == 8) dft8<DIR>(v);
    else if constexpr (R == 12) dft12<DIR>(v);
    else if constexpr (R == 16) dft16<DIR>(v);
}

// One in-place Stockham stage of radix R at span NS over B transforms, NT threads.
template <int N, int R, int NS, int DIR, int B, int BP, int NT>
__device__ __forceinline__ void stage(float2* __restrict__ buf, const float2* __restrict__ tw) {
    constexpr int kThreads = NT;
    constexpr int NB = N / R;
    constexpr int ITEMS = NB * B;
    constexpr int K = (ITEMS + kThreads - 1) / kThreads;
    float2 v[K][R];
#pragma unroll
    for (int it = 0; it < K; ++it) {
        const int e = threadIdx.x + it * kThreads;
        if (ITEMS % kThreads == 0 || e < ITEMS) {
            const int b = e % B, j = e / B;
#pragma unroll
            for (int r = 0; r < R; ++r) v[it][r] = buf[(j + r * NB) * BP + b];
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < K; ++it) {
        const int e = threadIdx.x + it * kThreads;
        if (ITEMS % kThreads == 0 || e < ITEMS) {
            const int b = e % B, j = e / B;
            const int k = j % NS;
            if constexpr (NS > 1) {
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    float2 w = tw[r * k * (N / (NS * R))];
                    if (DIR > 0) w.y = -w.y;
                    v[it][r] = cmul(v[it][r], w);
                }
            }
            dft<R, DIR>(v[it]);
            const int base = (j / NS) * NS * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) buf[(base + r * NS) * BP + b] = v[it][r];
        }
    }
    __syncthreads();
}

// Full length-N transform of the B transforms held in buf (natural order).
template <int N, int DIR, int B, int BP, int NT = kThreads>
__device__ __forceinline__ void fft_smem(float2* __restrict__ buf, const float2* __restrict__ tw) {
    using P = Plan<N>;
    stage<N, P::R0, 1, DIR, B, BP, NT>(buf, tw);
    if constexpr (P::R1 > 1) stage<N, P::R1, P::R0, DIR, B, BP, NT>(buf, tw);
    if constexpr (P::R2 > 1) stage<N, P::R2, P::R0 * P::R1, DIR, B, BP, NT>(buf, tw);
}

// threads of a column-pass CTA: eight elements of the N x CW tile per thread (16 at N = 512)
__host__ __device__ constexpr int col_threads_of(int n) {
    return (n * cw_of(n)) / 8 < 64 ? 64 : ((n * cw_of(n)) / 8 > 512 ? 512 : (n * cw_of(n)) / 8);
}

// Symmetric-wedge index of a sorted triple a <= b <= c: C(c+2,3) + C(b+1,2) + a.
__host__ __device__ __forceinline__ long long wedge_index(int a, int b, int c) {
    return (long long)c * (c + 1) * (c + 2) / 6 + (long long)b * (b + 1) / 2 + a;
}
__device__ __forceinline__ void sort3(int& a, int& b, int& c) {
    int t;
    if (a > b) { t = a; a = b; b = t; }
    if (b > c) { t = b; b = c; c = t; }
    if (a > b) { t = a; a = b; b = t; }
}
// Wedge index of an arbitrary (p, q, r) on an N grid (fold to [0, N/2], sort).
__device__ __forceinline__ long long wedge_of(int p, int q, int r, int n) {
    int a = p <= n - p ? p : n - p;
    int b = q <= n - q ? q : n - q;
    int c = r <= n - r ? r : n - r;
    sort3(a, b, c);
    return wedge_index(a, b, c);
}

} // namespace lc
