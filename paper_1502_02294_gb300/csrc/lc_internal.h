// lc_internal.h -- host planner and device-kernel launchers shared by the
// translation units of liblc (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/lc.h"

namespace lc {

// Kernels launched by the library in this process (lc_kernel_launches);
// every launch site adds its count here.
void count_launch(unsigned long long k = 1);

// ---------------- host FP64 planner (lc_host.cpp) ----------------
struct Cosmo {
    double om, h;
};
double hubble(const Cosmo& c, double z);                // km/s/Mpc
double chi(const Cosmo& c, double z1, double z2);       // comoving Mpc, Eq. 6
double time_myr(const Cosmo& c, double z);              // cosmic time, closed form
double z_of_time(const Cosmo& c, double t_myr);
double zs_of_r(const Cosmo& c, double z_obs, double r); // chi(z_obs, z_s) = r
double alpha_lw(const Cosmo& c, double zs);             // Eq. 16
double fmod_lw(double r, double alpha);                 // Eq. 15
// the radial kernel (LC_KERNEL_*): g(r) = (1+z_obs)^3 f(r, z_s) / ((4 pi)^2 (1+z_s) r^2)
// kKernelLwRough: the LW kernel with the rough horizon of Section 1
// (LC_KERNEL_LW with LC_HORIZON_ROUGH)
constexpr int kKernelLwRough = 2;
struct Kernel {
    int kind = LC_KERNEL_LW;
    double length = 0, rmax = 0; // LC_KERNEL_EXP: f = exp(-r / length) for r < rmax
};
double rough_horizon(double zs); // 100 [21 / (1 + z_s)]^0.5 Mpc (Section 1)
double kernel_f(const Cosmo& c, const Kernel& k, double zs, double r);
double horizon(const Cosmo& c, const Kernel& k, double z_obs); // LW: r / alpha(z_s(r)) = 97.39
double shell_integral(const Cosmo& c, const Kernel& k, double z_obs, double r_lo, double r_hi, double r_h);
int step_edges(const Cosmo& c, const Kernel& k, const lc_steps& st, std::vector<double>& z);
// g(r) at r = delta sqrt(8 t + 3), t < ntab
void g_table(const Cosmo& c, const Kernel& k, double z_obs, double delta, long long ntab, double* out);

struct StepGeom {
    int A = 0;                 // active slices (lookback j = 0 .. A-1)
    std::vector<double> lo, hi, I;
    double rh = 0;
    std::vector<long long> bnd; // A + 1 integer shell boundaries in units of delta^2
    long long Rh = 0;           // largest admissible R inside the horizon
    long long ntab = 0;
};
// cap > 0: at most cap lookback slices (the newest)
StepGeom step_geometry(const Cosmo& c, const Kernel& k, const std::vector<double>& z, int s, double l, int S,
                       bool integrals, int cap = 0);

// ---------------- device kernels (lc_device.cu) ----------------
struct SlotMeta {
    int slot, step;
    int* slot_step;
    double* slot_S;
    long long* slot_total;
    // optional (nullptr: none): the push counter, advanced by the source
    // check, and per grid row (x N + y) the counter value of the last push
    // that deposited into it, so that the z pass can skip rows left all zero
    unsigned* stamp;
    unsigned* rowstamp;
};
// Checks the luminosities (finite, >= 0; a bad one sets *err) and records the
// bits of their maximum; marks the slot (step, total = 0) and advances the
// push counter.
void launch_src_prep(const double* pos, const double* lum, long long n, unsigned long long* maxbits, int* err,
                     SlotMeta m, cudaStream_t st);
// Fixed-point deposit (LC_DEPOSIT_NGP or LC_DEPOSIT_CIC) into grid (int64,
// pre-zeroed), total into slot_total; a source with a non-finite position or
// luminosity, or a negative one, is left out and sets *err.  cell_out / q_out
// (may be null): the flat cell index and integer share of each of a source's
// cells (1 for NGP, 8 for CIC, at [cells * i + k]), kept for the near-field
// correction of the innermost shell; off_out (NGP only): each source's
// position relative to its cell centre.  With m.rowstamp, every row that
// receives a non-zero share is stamped with the push counter.
void launch_deposit(const double* pos, const double* lum, long long n, int N, double l, int deposit,
                    const unsigned long long* maxbits, long long* grid, SlotMeta m, int* err, cudaStream_t st,
                    long long* cell_out = nullptr, long long* q_out = nullptr, double* off_out = nullptr);

// Near field of the innermost shell (displacements |d|_inf <= R), which the
// FFT path leaves out: gnear holds the shell's FP64 values on the wedge prefix
// c <= R (kNearR, defined with the kernels).  prep: gnear from the builder's
// wedge, and the far part's k = 0 value.
void launch_near_prep(const double* gw0, const double* scale0, double* gnear, double* g0_far, cudaStream_t st);
// sub-cell near field of the innermost shell from the sources' own positions
struct NearPmArgs {
    const long long* cell;  // NGP cells of the sources
    const long long* q;     // fixed-point charges
    const double* off;      // positions relative to the cell centres (3 per source)
    long long n;
    int N, S, U;            // grid, sub-samples per axis, periodic images per axis (-U..U)
    double l, L;            // cell and box side
    double rtop;            // min(shell outer radius, horizon): the z_s table's range
    double rhi, rh;         // shell outer radius, horizon (FP64 decisions)
    float rtop2f;           // rtop^2 in FP32
    float win2f;            // |r^2 - rtop^2| <= win2f: decide the sample in FP64
    float prune2f;          // |c|^2 above this: no sample of the image reaches rtop
    // at r = k rtop / (K - 1): x = (1 + z_obs)^3 / ((4 pi)^2 (1 + z_s(r))),
    // y = 1 / (116.29 alpha(z_s(r))) for the LW kernel (Eq. 16), else 0
    const float2* tab;
    int K;
    int kind;               // radial kernel (LC_KERNEL_*, or kKernelLwRough)
    float xcut;             // LW kernels: f = 0 where r / (116.29 alpha) > xcut (Eq. 15's cut; none for the rough horizon)
    float inv_klen, kmax;   // LC_KERNEL_EXP parameters: 1 / length, cut-off
    const double* f0;       // the shell's normalisation factor (device)
    const double* slot_S;
    int slot;
    double U_out;
};
void launch_near_pm(const NearPmArgs& a, double* acc, cudaStream_t st);
// copy n4 float4 from device memory to the device view of page-locked host memory
void launch_copy_out(long long n4, const float4* src, float4* dst, int ctas, cudaStream_t st);
// sum over the A shells of a step's Ghat table ([W][gstride] FP32, summed in
// FP64 and rounded once) into column 0 of gsum [W][8] (other columns 0), and
// of the FP64 k = 0 values g0[A] into *g0sum
void launch_gsum(long long W, int A, int gstride, const float* ghat, const double* g0, float* gsum, double* g0sum,
                 cudaStream_t st);
// scatter U * S * q * G(d) into the FP64 accumulator for every source and d
// (NearScatter: the list and its factors, defined with the kernels)
struct NearScatter;
void launch_near_scatter(const NearScatter& a, int N, cudaStream_t st);
// fold the accumulator into out (one rounding per cell) and clear it; with a
// grid, also zero each entry's own deposit cell there (the sparse clear of the
// deposit grid, once the transforms have read it)
void launch_near_fold(const long long* cell, const long long* q, long long n, int N, double* acc, float* out,
                      long long* grid, cudaStream_t st);
// zero grid[cell[i]] for the n entries of a near-field list with q[i] != 0
void launch_cells_clear(const long long* cell, const long long* q, long long n, long long* grid, cudaStream_t st);

struct RgfAccumArgs {
    int N, S, A, U;
    double l;
    long long W;
    const long long* bnd;
    long long Rh;
    const double* gtab;
    double* gw; // [A][W]
    double rh;
};
void launch_rgf_accum(const RgfAccumArgs& a, cudaStream_t st);
// f_diff = (J_instant - J) / J per cell (Section 3 after Eq. 18)
void launch_fdiff(long long n, const float* j, const float* j_inst, float* out, cudaStream_t st);
// per shell: full-grid sum with multiplicities -> scale (normalisation) and Ghat(0)
void launch_rgf_norm(int N, long long W, int A, const double* gw, const double* I, double l3, int normalise,
                     double* scale, double* g0, cudaStream_t st);

} // namespace lc
