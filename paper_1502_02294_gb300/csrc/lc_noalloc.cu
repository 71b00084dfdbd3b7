// lc_noalloc.cu -- an allocation-free variant of lc_fft_r2c.
//
// Some callers cannot allocate device memory at the moment they want a
// transform: code running inside a memory pool that owns every byte of the
// device, a plug-in whose host forbids cudaMalloc (or where cudaMalloc would
// synchronise the device), or a latency-critical loop that must not pay an
// allocation.  lc_fft_r2c needs a padded work spectrum and a twiddle table
// and allocates them per call; lc_fft_r2c_static takes both from one
// file-scope device array instead and calls no cudaMalloc / cudaFree.
//
// The array below is part of the library image: every GPU on which the
// library is used keeps kStaticScratchBytes of device memory reserved for it
// until the process exits.  Its device address is obtained with
// cudaGetSymbolAddress once per device and CUDA context (the host-side name is
// only a stand-in and must never be passed to a kernel).  The cache is keyed
// on the context's unique ID as well as the device, so a context rebuilt by
// cudaDeviceReset (which reloads the module and may move the array) gets its
// own lookup instead of a stale address.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "lc_internal.h"
#include "lc_kernels.cuh"

namespace lc {
const FftOps* fft_ops_for(int n);
cudaError_t fft_ensure_init(const FftOps* ops);

namespace {

constexpr size_t kStaticScratchBytes = 4u << 20; // 4 MiB: grids up to N = 96
static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};
unsigned long long g_scratch_ctx[kMaxDevices] = {0}; // context ID the address belongs to

// The unique ID of the calling thread's current context (0 if none or if the
// driver does not offer it), through the driver entry points the runtime
// hands out, so the library needs no link against the driver library.
unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        looked_up = true;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void**)&get_current, 12000, cudaEnableDefault, &q1) !=
                cudaSuccess || q1 != cudaDriverEntryPointSuccess)
            get_current = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", (void**)&get_id, 12000, cudaEnableDefault, &q2) !=
                cudaSuccess || q2 != cudaDriverEntryPointSuccess)
            get_id = nullptr;
        cudaGetLastError();
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

__global__ void k_twiddles(float2* tw, int n) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < n) {
        double s, c;
        sincospi(2.0 * m / n, &s, &c);
        tw[m] = make_float2((float)c, (float)-s);
    }
}

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

} // namespace
} // namespace lc

using namespace lc;

extern "C" lc_status lc_fft_r2c_static(int n, const float* in, float* out_complex, void* stream) {
    if (!in || !out_complex) return LC_ERR_INVALID_ARG;
    const FftOps* ops = fft_ops_for(n);
    if (!ops) return LC_ERR_UNSUPPORTED_SIZE;
    const size_t work_bytes = sizeof(float2) * (size_t)n * n * nrp_of(n);
    if (round256(work_bytes) + sizeof(float2) * n > kStaticScratchBytes) return LC_ERR_UNSUPPORTED_SIZE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return LC_ERR_CUDA;
    }
    void* base = nullptr;
    {
        // first call on this device (or in a new context of it): resolve the
        // array's device address in the current context
        std::lock_guard<std::mutex> g(g_mu);
        const unsigned long long ctx = current_context_id();
        if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
            void* addr = nullptr;
            if (cudaGetSymbolAddress(&addr, g_scratch) != cudaSuccess || !addr) {
                g_scratch_addr[dev] = nullptr;
                cudaGetLastError();
                return LC_ERR_CUDA;
            }
            g_scratch_addr[dev] = addr;
            g_scratch_ctx[dev] = current_context_id(); // the lookup made the primary context current if none was
        }
        base = g_scratch_addr[dev];
    }
    if (fft_ensure_init(ops) != cudaSuccess) return LC_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    float2* work = static_cast<float2*>(base);
    float2* tw = reinterpret_cast<float2*>(static_cast<unsigned char*>(base) + round256(work_bytes));
    // every call rewrites the twiddles and every element of the work
    // spectrum it later reads, so nothing left by an earlier call is used
    k_twiddles<<<(n + 127) / 128, 128, 0, st>>>(tw, n);
    RowR2CArgs ra{};
    ra.in_mode = ROW_IN_F32;
    ra.nrows = (long long)n * n;
    ra.fin = in;
    ra.dst = work;
    ra.tw = tw;
    ColArgs c{};
    c.axis = 0;
    c.dir = -1;
    c.in_mode = COL_IN_PLAIN;
    c.out_mode = COL_OUT_PLAIN;
    c.src = work;
    c.dst = work;
    c.tw = tw;
    const bool pl = ops->plane_r2c && ops->plane_on();
    if (pl) {
        ops->plane_r2c(ra, st);
    } else {
        ops->rows_r2c(ra, st);
        ops->cols(c, st);
    }
    c.axis = 1;
    ops->cols(c, st);
    const int h = n / 2 + 1;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) count_launch(pl ? 3 : 4); // twiddles + the transform's passes
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(out_complex, sizeof(float2) * h, work, sizeof(float2) * nrp_of(n), sizeof(float2) * h,
                              (size_t)n * n, cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? LC_OK : LC_ERR_CUDA;
}
