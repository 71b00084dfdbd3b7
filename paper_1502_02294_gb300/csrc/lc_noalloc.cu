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
// until the process exits.  Its device address is obtained once per device
// with cudaGetSymbolAddress (the host-side name is only a stand-in and must
// never be passed to a kernel).
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
        // first call on this device: resolve the array's device address
        std::lock_guard<std::mutex> g(g_mu);
        if (!g_scratch_addr[dev]) {
            if (cudaGetSymbolAddress(&g_scratch_addr[dev], g_scratch) != cudaSuccess) {
                g_scratch_addr[dev] = nullptr;
                cudaGetLastError();
                return LC_ERR_CUDA;
            }
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
    if (ops->plane_r2c) {
        ops->plane_r2c(ra, st);
    } else {
        ops->rows_r2c(ra, st);
        ops->cols(c, st);
    }
    c.axis = 1;
    ops->cols(c, st);
    const int h = n / 2 + 1;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(out_complex, sizeof(float2) * h, work, sizeof(float2) * nrp_of(n), sizeof(float2) * h,
                              (size_t)n * n, cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? LC_OK : LC_ERR_CUDA;
}
