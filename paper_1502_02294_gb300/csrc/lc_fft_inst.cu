// lc_fft_inst.cu -- instantiates the FFT pass kernels for one grid size.
// Compiled once per supported N with -DLC_N=<N> (separate objects, built in
// parallel); each object exports the launcher table lc_fft_ops_<N>.
#include "lc_mac.cuh"

#ifndef LC_N
#error "LC_N must be defined"
#endif
#define LC_CAT2(a, b) a##b
#define LC_CAT(a, b) LC_CAT2(a, b)

namespace lc {
namespace {
cudaError_t init_all() {
    cudaError_t e = Launch<LC_N>::init();
    if (e == cudaSuccess) e = MacLaunch<LC_N, false>::init();
    if (e == cudaSuccess) e = MacLaunch<LC_N, true>::init();
    if (e == cudaSuccess) e = MacWsLaunch<LC_N, false, false>::init();
    if (e == cudaSuccess) e = MacWsLaunch<LC_N, true, false>::init();
    if (e == cudaSuccess) e = MacWsLaunch<LC_N, false, true>::init();
    if (e == cudaSuccess) e = MacWsLaunch<LC_N, true, true>::init();
    return e;
}
void mac_f32(const MacArgs& a, cudaStream_t st) { MacLaunch<LC_N, false>::run(a, st); }
void mac_bf16(const MacArgs& a, cudaStream_t st) { MacLaunch<LC_N, true>::run(a, st); }
void mac_ws_f32(const MacArgs& a, cudaStream_t st) { MacWsLaunch<LC_N, false, false>::run(a, st); }
void mac_ws_bf16(const MacArgs& a, cudaStream_t st) { MacWsLaunch<LC_N, true, false>::run(a, st); }
void mac_ws2_f32(const MacArgs& a, cudaStream_t st) { MacWsLaunch<LC_N, false, true>::run(a, st); }
void mac_ws2_bf16(const MacArgs& a, cudaStream_t st) { MacWsLaunch<LC_N, true, true>::run(a, st); }
} // namespace
extern const FftOps LC_CAT(fft_ops_, LC_N);
const FftOps LC_CAT(fft_ops_, LC_N) = {LC_N,
                                      &init_all,
                                      &Launch<LC_N>::rows_r2c,
                                      &Launch<LC_N>::cols,
                                      &Launch<LC_N>::rows_c2r,
                                      (plane_ok<LC_N>() || plane_cl_ok<LC_N>()) ? &Launch<LC_N>::plane_r2c : nullptr,
                                      (plane_ok<LC_N>() || plane_cl_ok<LC_N>()) ? &Launch<LC_N>::plane_c2r : nullptr,
                                      MacCfg<LC_N, false>::OK ? &mac_f32 : nullptr,
                                      MacCfg<LC_N, true>::OK ? &mac_bf16 : nullptr,
                                      MacWsCfg<LC_N, false, false>::OK ? &mac_ws_f32 : nullptr,
                                      MacWsCfg<LC_N, true, false>::OK ? &mac_ws_bf16 : nullptr,
                                      MacWsCfg<LC_N, false, true>::OK ? &mac_ws2_f32 : nullptr,
                                      MacWsCfg<LC_N, true, true>::OK ? &mac_ws2_bf16 : nullptr,
                                      LC_N * Launch<LC_N>::NCH,
                                      &Launch<LC_N>::variants_built,
                                      &Launch<LC_N>::set_variant,
                                      &Launch<LC_N>::get_variant,
                                      &Launch<LC_N>::plane_near_ctas,
                                      &Launch<LC_N>::plane_on,
                                      plane_cl_ok<LC_N>()};
} // namespace lc
