// lc_fft_inst.cu -- instantiates the FFT pass kernels for one grid size.
// Compiled once per supported N with -DLC_N=<N> (separate objects, built in
// parallel); each object exports the launcher table lc_fft_ops_<N>.
#include "lc_kernels.cuh"

#ifndef LC_N
#error "LC_N must be defined"
#endif
#define LC_CAT2(a, b) a##b
#define LC_CAT(a, b) LC_CAT2(a, b)

namespace lc {
extern const FftOps LC_CAT(fft_ops_, LC_N);
const FftOps LC_CAT(fft_ops_, LC_N) = {LC_N, &Launch<LC_N>::init, &Launch<LC_N>::rows_r2c, &Launch<LC_N>::cols,
                                      &Launch<LC_N>::rows_c2r};
} // namespace lc
