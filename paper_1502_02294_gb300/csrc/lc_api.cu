// lc_api.cu -- the C ABI of liblc (see include/lc.h): plan lifecycle, the
// per-step orchestration of the hot path, the per-observing-step Green's
// function tables, and stand-alone kernel entry points.
//
// Per step (all on the plan's stream):
//   push  : memset(grid) -> src_prep -> deposit -> rows r2c (int64 in)
//           -> y-pass -> x-pass with ring-slot epilogue         (step 4, Sec. 2.2)
//   field : x-pass with shell-MAC prologue (+ FP64 k = 0) -> y-pass
//           -> rows c2r with U / N^3 epilogue                   (steps 5-6)
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <new>
#include <vector>

#include "lc_internal.h"
#include "lc_mac.cuh"

namespace lc {
extern const FftOps fft_ops_8, fft_ops_16, fft_ops_32, fft_ops_64, fft_ops_96, fft_ops_128, fft_ops_192,
    fft_ops_256, fft_ops_384, fft_ops_512;

const FftOps* fft_ops_for(int n);
static const FftOps* ops_for(int n) { return fft_ops_for(n); }
const FftOps* fft_ops_for(int n) {
    switch (n) {
    case 8: return &fft_ops_8;
    case 16: return &fft_ops_16;
    case 32: return &fft_ops_32;
    case 64: return &fft_ops_64;
    case 96: return &fft_ops_96;
    case 128: return &fft_ops_128;
    case 192: return &fft_ops_192;
    case 256: return &fft_ops_256;
    case 384: return &fft_ops_384;
    case 512: return &fft_ops_512;
    default: return nullptr;
    }
}

// cudaFuncSetAttribute once per (device, N)
cudaError_t fft_ensure_init(const FftOps* ops);
static cudaError_t ensure_init(const FftOps* ops) { return fft_ensure_init(ops); }
cudaError_t fft_ensure_init(const FftOps* ops) {
    static std::mutex mu;
    static std::vector<std::pair<int, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> g(mu);
    for (auto& d : done)
        if (d.first == dev && d.second == ops->n) return cudaSuccess;
    e = ops->init();
    if (e == cudaSuccess) done.push_back({dev, ops->n});
    return e;
}

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// The device address of page-locked host memory (null for any other pointer).
static void* pinned_device_view(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

static int sm_count() {
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

// ---- tensor maps of the TMA column passes ----
// cuTensorMapEncodeTiled through the driver entry point the runtime hands out
// (no link against the driver library)
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static bool looked_up = false;
    static std::mutex mu;
    std::lock_guard<std::mutex> g(mu);
    if (!looked_up) {
        looked_up = true;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void**)&fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess || q != cudaDriverEntryPointSuccess)
            fn = nullptr;
        cudaGetLastError();
    }
    return fn;
}

// The half spectrum at `work` ([p][q][NRP complex], C order) as a rank-3
// tensor of floats (2 NRP, N, N), with the box of one column-pass tile: CW
// columns by N (from 384: N / 2) lines q of one plane p (y pass, axis 0), or
// CW columns by as many planes p of one line q (x pass, axis 1).
bool make_cols_map(CUtensorMap* m, const float2* work, int n, int axis) {
    EncodeTiledFn fn = encode_tiled();
    if (!fn || (reinterpret_cast<uintptr_t>(work) & 15)) return false;
    const cuuint64_t nrp = (cuuint64_t)nrp_of(n), N = (cuuint64_t)n;
    const cuuint32_t cw = (cuuint32_t)cw_of(n), box_t = n > 256 ? (cuuint32_t)(n / 2) : (cuuint32_t)n;
    const cuuint64_t dims[3] = {2 * nrp, N, N};
    const cuuint64_t strides[2] = {nrp * sizeof(float2), N * nrp * sizeof(float2)};
    const cuuint32_t box[3] = {2 * cw, axis == 0 ? box_t : 1u, axis == 0 ? 1u : box_t};
    const cuuint32_t es[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2*>(work), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The two maps of a work spectrum (y and x pass), made where a TMA form exists for n.
struct ColsMaps {
    CUtensorMap y, x;
    bool ok = false;
    void make(const float2* work, int n) {
        const FftOps* ops = fft_ops_for(n);
        ok = ops && (ops->cols_variants() >> FFT_COLS_TMA & 1) && make_cols_map(&y, work, n, 0) &&
             make_cols_map(&x, work, n, 1);
    }
    // a plain column pass over the spectrum these maps describe: its map by axis
    void set(ColArgs& c, int* err) const {
        c.tmap = ok ? (c.axis == 0 ? &y : &x) : nullptr;
        c.err = err;
    }
};

static std::vector<float2> twiddles(int n) {
    std::vector<float2> t(n);
    for (int m = 0; m < n; ++m) {
        const double a = 2.0 * 3.141592653589793238462643383279502884 * m / n;
        t[m] = make_float2((float)cos(a), (float)-sin(a));
    }
    return t;
}

static std::atomic<unsigned long long> g_launches{0};
void count_launch(unsigned long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

} // namespace lc

using namespace lc;

// ---------------------------------------------------------------- autotuner
// The shell MAC has four variants: a register-gather pass (MAC_GATHER), a
// bulk-copy pipelined kernel for the full tiles (MAC_BULK), and its
// warp-specialised form over every tile, one tile per CTA (MAC_WS) or the
// tiles of lines q and N - q together (MAC_WS2).  Which one is fastest
// depends on the grid, the history precision and the number of active
// slices; the plan times each on its own buffers the first time it meets a
// (device, N, history, slices) combination and keeps the fastest.  Choices
// are kept per process and, when LC_AUTOTUNE_CACHE names a file, loaded
// from and appended to that file.  LC_MAC_VARIANT=gather|bulk|ws|ws2 forces
// one variant where it is built (tests).
enum { MAC_GATHER = 0, MAC_BULK = 1, MAC_WS = 2, MAC_WS2 = 3, MAC_NVAR = 4 };
const char* const kMacNames[MAC_NVAR] = {"gather", "bulk", "ws", "ws2"};
namespace {
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;
bool g_tune_loaded = false;
std::map<int, int> g_fft_forced; // grid size -> FFT variant forced by lc_fft_set_variant

void tune_load() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char* path = getenv("LC_AUTOTUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    // one choice per line: key, variant, then the measured times (ignored)
    char line[512], key[256];
    int v;
    while (fgets(line, sizeof line, f))
        if (sscanf(line, "%255s %d", key, &v) == 2 && v >= 0 && v < 16) g_tune[key] = v; // range checked at use
    fclose(f);
}

void tune_store(const std::string& key, int v, const double* ms, int nms) {
    g_tune[key] = v;
    const char* path = getenv("LC_AUTOTUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d", key.c_str(), v);
    for (int i = 0; i < nms; ++i) fprintf(f, " %.6f", ms[i]);
    fprintf(f, "\n");
    fclose(f);
}
} // namespace

struct lc_plan {
    int N = 0;
    double L = 0, l = 0;
    Cosmo cosmo{0, 0};
    Kernel kern;
    int n_steps = 0, S = 4, history = 0, normalise = 1;
    int deposit = LC_DEPOSIT_NGP; // source assignment (LC_DEPOSIT_*)
    int n_shell_max = 0;          // > 0: at most this many lookback slices per step
    double U = 1.0;
    std::vector<double> z;
    cudaStream_t stream = nullptr;
    const FftOps* ops = nullptr;
    int NRP = 0;
    long long spec_elems = 0, W = 0;
    std::vector<int> A_of_step;
    int n_ring = 1;
    // device state
    long long* d_grid = nullptr;
    float2* d_work = nullptr;
    void* d_ring = nullptr;
    int* d_slot_step = nullptr;
    double* d_slot_S = nullptr;
    long long* d_slot_total = nullptr;
    float2* d_tw = nullptr;
    ColsMaps maps; // tensor maps of d_work for the TMA column passes
    int* d_err = nullptr;
    unsigned long long* d_maxbits = nullptr;
    // push counter and, per grid row, the counter of its last deposit (the
    // z pass skips rows without a share of the current push)
    unsigned* d_stamp = nullptr;
    unsigned* d_rowstamp = nullptr;
    double* d_pos = nullptr;
    double* d_lum = nullptr;
    long long src_cap = 0;
    float* d_out_stage = nullptr;
    // asynchronous host output (lc_retarded_field_async): two device stages,
    // each copied out on a copy stream while the next step computes
    cudaStream_t copy_stream = nullptr;
    float* d_out_async[2] = {nullptr, nullptr};
    cudaEvent_t ev_computed[2] = {nullptr, nullptr}, ev_copied[2] = {nullptr, nullptr};
    uint64_t tickets = 0;              // tickets issued; ticket t used stage (t - 1) % 2
    uint64_t stage_ticket[2] = {0, 0}; // the last ticket of each stage
    // completion of each ticket's copy: its own event (a ring of kTicketEvents,
    // re-recorded only kTicketEvents tickets later), and the highest ticket
    // known complete (copies complete in ticket order on the one copy stream)
    static constexpr int kTicketEvents = 16;
    cudaEvent_t ev_ticket[kTicketEvents] = {};
    uint64_t done_upto = 0;
    // Green's function tables, one per observing step (built lazily)
    long long ring_slot = 0; // complex elements per tile-major ring slot: N^2 (N/2 + 1)
    struct Table {
        int gstride = 0;        // row stride of ghat: A rounded up to 8
        float* ghat = nullptr;  // [W][gstride]; shell 0 without its near cube when near_on
        double* g0 = nullptr;   // [A] FP64 Ghat_j(0) of what the FFT path carries
        double* gnear = nullptr; // near cube of shell 0 on the wedge prefix (near_on)
        float2* pmtab = nullptr; // near_pm: the redshift factors of g on [0, rtop] (kZsTab points)
        double rtop = 0, rhi0 = 0, rh = 0;
        int mac_variant = 0;    // MAC_GATHER, MAC_BULK, MAC_WS or MAC_WS2, chosen by the autotuner
        int A = -1;             // -1: not built
        // the instantaneous field (Eq. 18) sees one slice through every shell:
        // sum_j Ghat_j as a one-shell table [W][8] and sum_j Ghat_j(0) in FP64,
        // built on the first lc_instant_field of the step
        float* gsum = nullptr;
        double* g0sum = nullptr;
        int inst_variant = 0;
    };
    std::vector<Table> tables;
    // table budget: 0 = keep every table; else tables of other observing
    // steps are freed (oldest first) to keep the total under it
    size_t table_budget = 0, table_bytes = 0;
    std::vector<int> table_pins; // per step: > 0 while a graph holds its table
    // builder scratch
    double* d_gw = nullptr;
    long long gw_cap = 0;
    double* d_gtab = nullptr;
    long long gtab_cap = 0;
    long long* d_bnd = nullptr;
    double* d_I = nullptr;
    double* d_scale = nullptr;
    // autotuner scratch: slot tables marking every slice valid
    int* d_tune_step = nullptr;
    double* d_tune_S = nullptr;
    long long* d_tune_total = nullptr;
    // near field of the innermost shell, added exactly (FP32 history)
    bool near_on = false;
    double* d_near = nullptr;     // N^3 FP64 accumulator, kept all-zero between steps
    long long* d_src_cell = nullptr;
    long long* d_src_q = nullptr;
    bool near_pm = false;           // near cube from the sources' own positions
    double* d_src_off = nullptr;    // near_pm: positions relative to the cell centres (3 per source)
    long long near_cap = 0, near_n = 0;
    // near-field lists replaced by larger ones: a captured step graph may still
    // write and read them, so they stay allocated until the plan is destroyed
    std::vector<void*> retired;
    size_t bytes = 0;
    // the deposit grid holds the charges of the last push until its cells
    // are cleared; with a near-field list (near_on) only those cells are
    // zeroed (by the near fold of the step's field, or before the next
    // deposit when no field ran), never the whole grid
    bool grid_dirty = false;
    // inside lc_graph_create, whose field follows its push at once: the push
    // may leave its x pass into the ring to the field's gather MAC
    // (fuse_x), which then owes it for ring slot x_deferred
    bool fuse_x = false;
    int x_deferred = -1;
    int last_pushed = -1;
    bool failed = false;
    // per-phase event timing
    bool timing = false;
    struct Mark {
        int phase;
        cudaEvent_t a, b;
    };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> pool;
    double ms[LC_N_PHASES] = {0};
    long long launches[LC_N_PHASES] = {0};
    // graph capture of a whole step (lc_graph_create)
    bool capturing = false;
    long long cap_kernels[LC_N_PHASES] = {0};
    std::vector<lc_step_graph*> graphs;
};

struct lc_batch_graph {
    std::vector<lc_plan*> plans;
    std::vector<int> steps;
    std::vector<long long> n_src;
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;
};

struct lc_step_graph {
    lc_plan* p = nullptr;
    int step = 0;
    long long n_src = 0;
    cudaGraphExec_t exec = nullptr;
    std::vector<lc_plan::Mark> marks; // phase events inside the graph (timing on at capture)
    long long kernels[LC_N_PHASES] = {0};
    bool pending = false;             // replayed, events not yet read
};

namespace {

cudaEvent_t take_event(lc_plan* p) {
    if (!p->pool.empty()) {
        cudaEvent_t e = p->pool.back();
        p->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Scoped phase marker: records an event pair on the plan's stream when
// timing is on; always counts the phase's kernel launches.
struct Phase {
    lc_plan* p;
    int ph;
    int k;
    cudaEvent_t a = nullptr;
    // inside a stream capture the events must become event-record nodes
    // (external), not capture-internal dependencies
    void record(cudaEvent_t e) {
        if (p->capturing) cudaEventRecordWithFlags(e, p->stream, cudaEventRecordExternal);
        else cudaEventRecord(e, p->stream);
    }
    Phase(lc_plan* p_, int ph_, int kernels) : p(p_), ph(ph_), k(kernels) {
        if (p->timing) {
            a = take_event(p);
            record(a);
        }
    }
    ~Phase() {
        if (p->timing) {
            cudaEvent_t b = take_event(p);
            record(b);
            p->marks.push_back({ph, a, b});
        }
        if (p->capturing) {
            p->cap_kernels[ph] += k; // counted when the graph is launched
        } else {
            p->launches[ph] += k;
            count_launch(k);
        }
    }
};

// read the phase events of a graph's last replay into the plan's totals
void harvest_graph(lc_plan* p, lc_step_graph* g) {
    if (!g->pending) return;
    if (!g->marks.empty()) cudaEventSynchronize(g->marks.back().b);
    for (auto& m : g->marks) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, m.a, m.b) == cudaSuccess) p->ms[m.phase] += t;
        else cudaGetLastError();
    }
    g->pending = false;
}

lc_status cuda_fail(lc_plan* p, cudaError_t e) {
    if (e == cudaSuccess) return LC_OK;
    if (p) p->failed = true;
    return e == cudaErrorMemoryAllocation ? LC_ERR_OOM : LC_ERR_CUDA;
}

// z and y of a step's transforms by plane kernels (one launch each way): for
// grids up to 192^3 always, at 256^3 in the four-CTA cluster form when chosen
static bool plane_step(const lc_plan* p) { return p->ops->plane_r2c && p->ops->plane_on(); }
// the Green's function tables through plane kernels (one CTA per plane only)
static bool plane_table(const lc_plan* p) { return p->ops->plane_r2c && !p->ops->plane_clustered; }

template <class T> cudaError_t dalloc(lc_plan* p, T** ptr, size_t count) {
    *ptr = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)ptr, sizeof(T) * count);
    if (e == cudaSuccess) p->bytes += sizeof(T) * count;
    else cudaGetLastError();
    return e;
}

void free_all(lc_plan* p) {
    for (auto* g : p->graphs) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        for (auto& m : g->marks) {
            cudaEventDestroy(m.a);
            cudaEventDestroy(m.b);
        }
        delete g;
    }
    p->graphs.clear();
    cudaFree(p->d_grid);
    cudaFree(p->d_work);
    cudaFree(p->d_ring);
    cudaFree(p->d_slot_step);
    cudaFree(p->d_slot_S);
    cudaFree(p->d_slot_total);
    cudaFree(p->d_tw);
    cudaFree(p->d_err);
    cudaFree(p->d_maxbits);
    cudaFree(p->d_stamp);
    cudaFree(p->d_rowstamp);
    cudaFree(p->d_pos);
    cudaFree(p->d_lum);
    cudaFree(p->d_out_stage);
    if (p->copy_stream) cudaStreamSynchronize(p->copy_stream);
    for (int k = 0; k < 2; ++k) {
        cudaFree(p->d_out_async[k]);
        if (p->ev_computed[k]) cudaEventDestroy(p->ev_computed[k]);
        if (p->ev_copied[k]) cudaEventDestroy(p->ev_copied[k]);
    }
    for (auto& ev : p->ev_ticket)
        if (ev) cudaEventDestroy(ev);
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    cudaFree(p->d_gw);
    cudaFree(p->d_gtab);
    cudaFree(p->d_bnd);
    cudaFree(p->d_I);
    cudaFree(p->d_scale);
    cudaFree(p->d_near);
    cudaFree(p->d_tune_step);
    cudaFree(p->d_tune_S);
    cudaFree(p->d_tune_total);
    cudaFree(p->d_src_cell);
    cudaFree(p->d_src_q);
    cudaFree(p->d_src_off);
    for (void* r : p->retired) cudaFree(r);
    for (auto& t : p->tables) {
        cudaFree(t.ghat);
        cudaFree(t.g0);
        cudaFree(t.gnear);
        cudaFree(t.pmtab);
        cudaFree(t.gsum);
        cudaFree(t.g0sum);
    }
    for (auto& m : p->marks) {
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    for (auto e : p->pool) cudaEventDestroy(e);
}

bool valid_steps(const lc_steps* st) {
    if (!st || st->n_steps < 1 || st->n_steps > 100000) return false;
    if (st->subsamples != 0 && (st->subsamples < 2 || st->subsamples > 16 || st->subsamples % 2)) return false;
    if (st->history != LC_HISTORY_FP32 && st->history != LC_HISTORY_BF16) return false;
    if (!(st->out_unit >= 0.0) || !isfinite(st->out_unit)) return false;
    if (st->spacing == LC_STEPS_EQUAL_TIME && !(st->z_start > st->z_end && st->z_end >= 0.0)) return false;
    if (st->spacing == LC_STEPS_EQUAL_TAU && (st->n_shell < 1 || !(st->z_end >= 0.0))) return false;
    if (st->spacing == LC_STEPS_EXPLICIT && !st->z_edges) return false;
    if (st->kernel != LC_KERNEL_LW && st->kernel != LC_KERNEL_EXP) return false;
    if (st->near_mode != LC_NEAR_NGP && st->near_mode != LC_NEAR_SUBCELL && st->near_mode != LC_NEAR_NONE)
        return false;
    if (st->kernel == LC_KERNEL_EXP && !(st->kernel_length > 0.0 && isfinite(st->kernel_length) &&
                                         st->kernel_rmax > 0.0 && isfinite(st->kernel_rmax)))
        return false;
    if (st->deposit != LC_DEPOSIT_NGP && st->deposit != LC_DEPOSIT_CIC) return false;
    // the sub-cell near field replaces the near cube of a source's NGP cell
    if (st->deposit == LC_DEPOSIT_CIC && st->near_mode == LC_NEAR_SUBCELL) return false;
    if (st->horizon_mode != LC_HORIZON_EQ15 && st->horizon_mode != LC_HORIZON_ROUGH) return false;
    if (st->horizon_mode == LC_HORIZON_ROUGH && st->kernel != LC_KERNEL_LW) return false;
    if (st->n_shell_max < 0) return false;
    return st->spacing >= 0 && st->spacing <= 2;
}

Kernel kernel_of(const lc_steps* st) {
    Kernel k;
    k.kind = st->kernel == LC_KERNEL_LW && st->horizon_mode == LC_HORIZON_ROUGH ? kKernelLwRough : st->kernel;
    k.length = st->kernel_length;
    k.rmax = st->kernel_rmax;
    return k;
}

// entries of the near-field list per source: its one NGP cell, or its 8 CIC cells
long long near_entries(const lc_plan* p, long long n_src) {
    return p->near_on ? n_src * (p->deposit == LC_DEPOSIT_CIC ? 8 : 1) : 0;
}

// Zero the cells the last push deposited into, if a field has not done so
// yet (sparse clear: the plan keeps a near-field list); on stream st.
void clear_grid_cells(lc_plan* p, cudaStream_t st) {
    if (!p->grid_dirty) return;
    if (p->near_on) {
        launch_cells_clear(p->d_src_cell, p->d_src_q, p->near_n, p->d_grid, st);
        count_launch(1);
    }
    p->grid_dirty = false;
}

bool valid_cosmo(const lc_cosmology* c) {
    return c && c->omega_m > 0.0 && c->omega_m <= 1.0 && c->h > 0.0 && isfinite(c->h);
}

// The shell-MAC phase of one field evaluation (inverse x pass with the
// products summed over slices) in the given variant.
void launch_mac(lc_plan* p, const lc_plan::Table& T, int step, int instant, int variant, const int* slot_step,
                const double* slot_S, const long long* slot_total, cudaStream_t st) {
    const bool bf = p->history == LC_HISTORY_BF16;
    ColArgs c{};
    c.axis = 1;
    c.dir = 1;
    c.in_mode = bf ? COL_IN_MAC_BF16 : COL_IN_MAC_F32;
    c.out_mode = COL_OUT_PLAIN;
    c.dst = p->d_work;
    c.ring = p->d_ring;
    c.slot_elems = p->ring_slot;
    c.n_ring = p->n_ring;
    c.step = step;
    c.A = T.A;
    c.slot_step = slot_step;
    c.slot_S = slot_S;
    c.slot_total = slot_total;
    c.ghat = T.ghat;
    c.g0 = T.g0;
    c.gstride = T.gstride;
    c.instant = instant;
    c.tw = p->d_tw;
    if (p->x_deferred >= 0 && variant == MAC_GATHER && !instant) {
        // the push's x pass of the newest slice, done in this kernel
        c.in_mode = bf ? COL_IN_MAC_BF16_X : COL_IN_MAC_F32_X;
        c.src = p->d_work;
        c.ring_out = p->d_ring;
        c.wslot = p->x_deferred;
        p->x_deferred = -1;
    }
    auto mac_fn = variant == MAC_WS    ? (bf ? p->ops->mac_ws_bf16 : p->ops->mac_ws_f32)
                  : variant == MAC_WS2 ? (bf ? p->ops->mac_ws2_bf16 : p->ops->mac_ws2_f32)
                                       : (bf ? p->ops->mac_bf16 : p->ops->mac_f32);
    if (variant != MAC_GATHER && mac_fn) {
        // MAC_BULK: full tiles in the bulk-copy kernel, the Nyquist tiles in
        // the generic pass; MAC_WS, MAC_WS2: every tile in one kernel
        MacArgs ma{p->d_ring, p->ring_slot, step, T.A, T.gstride, p->n_ring, slot_step, slot_S,
                   slot_total, T.ghat, T.g0, p->d_work, p->d_tw, p->d_err, bf ? 1 : 0, instant};
        mac_fn(ma, st);
        if (variant == MAC_WS || variant == MAC_WS2) return;
        c.tile0 = p->ops->full_tiles;
    }
    p->ops->cols(c, st);
}

bool mac_built(const lc_plan* p, int variant) {
    const bool bf = p->history == LC_HISTORY_BF16;
    if (variant == MAC_BULK) return (bf ? p->ops->mac_bf16 : p->ops->mac_f32) != nullptr;
    if (variant == MAC_WS) return (bf ? p->ops->mac_ws_bf16 : p->ops->mac_ws_f32) != nullptr;
    if (variant == MAC_WS2) return (bf ? p->ops->mac_ws2_bf16 : p->ops->mac_ws2_f32) != nullptr;
    return true;
}

int mac_kernels(const lc_plan* p, int variant) { return variant == MAC_BULK && mac_built(p, variant) ? 2 : 1; }

// The autotuners' timing: a transient buffer of twice the L2 size whose
// memset before each timed launch evicts the launch's inputs, as the other
// passes of a step do (without it, grids whose data fits in L2 were timed
// warm and the choice flipped from process to process).
struct TuneFlush {
    void* buf = nullptr;
    size_t bytes = 0;
    TuneFlush() {
        int dev = 0, l2 = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess)
            l2 = 0;
        bytes = 2 * (size_t)l2;
        if (bytes && cudaMalloc(&buf, bytes) != cudaSuccess) buf = nullptr;
        cudaGetLastError();
    }
    ~TuneFlush() {
        if (buf) cudaFree(buf);
    }
    TuneFlush(const TuneFlush&) = delete;
    TuneFlush& operator=(const TuneFlush&) = delete;
};

// Median time of `launch` (ms) over kTuneReps launches, each after an L2
// flush and between its own pair of events, after one warm-up; -1 on error.
constexpr int kTuneReps = 7;
template <class F> double tune_time(cudaStream_t st, const TuneFlush& fl, F&& launch) {
    cudaEvent_t a[kTuneReps] = {}, b[kTuneReps] = {};
    bool ok = true;
    for (int r = 0; ok && r < kTuneReps; ++r)
        ok = cudaEventCreate(&a[r]) == cudaSuccess && cudaEventCreate(&b[r]) == cudaSuccess;
    double med = -1.0;
    if (ok) {
        launch();
        for (int r = 0; r < kTuneReps; ++r) {
            if (fl.buf) cudaMemsetAsync(fl.buf, 0, fl.bytes, st);
            cudaEventRecord(a[r], st);
            launch();
            cudaEventRecord(b[r], st);
        }
        if (cudaEventSynchronize(b[kTuneReps - 1]) == cudaSuccess) {
            float t[kTuneReps];
            for (int r = 0; r < kTuneReps; ++r) {
                t[r] = 0.f;
                cudaEventElapsedTime(&t[r], a[r], b[r]);
            }
            std::sort(t, t + kTuneReps);
            med = t[kTuneReps / 2];
        }
    }
    for (int r = 0; r < kTuneReps; ++r) {
        if (a[r]) cudaEventDestroy(a[r]);
        if (b[r]) cudaEventDestroy(b[r]);
    }
    cudaGetLastError();
    return med;
}

// Pick the MAC variant for a table (plan time: may synchronise).
int choose_mac_variant(lc_plan* p, const lc_plan::Table& T, int s) {
    const bool bf = p->history == LC_HISTORY_BF16;
    if (const char* f = getenv("LC_MAC_VARIANT")) {
        for (int v = 0; v < MAC_NVAR; ++v)
            if (!strcmp(f, kMacNames[v])) return mac_built(p, v) ? v : MAC_GATHER;
    }
    int nbuilt = 0;
    for (int v = 1; v < MAC_NVAR; ++v) nbuilt += mac_built(p, v);
    if (!nbuilt) return MAC_GATHER;
    int dev = 0, major = 0, minor = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    char kb[128];
    snprintf(kb, sizeof kb, "mac%dc/sm%d%d/N%d/%s/A%d", MAC_NVAR, major, minor, p->N, bf ? "bf16" : "fp32", T.A);
    const std::string key(kb);
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        tune_load();
        auto it = g_tune.find(key);
        if (it != g_tune.end() && it->second < MAC_NVAR && mac_built(p, it->second)) return it->second;
    }
    // time every built variant with every slice marked valid (the ring's
    // contents do not matter for timing; the output goes to the work buffer)
    if (!p->d_tune_step) {
        if (dalloc(p, &p->d_tune_step, p->n_ring) != cudaSuccess || dalloc(p, &p->d_tune_S, p->n_ring) != cudaSuccess ||
            dalloc(p, &p->d_tune_total, p->n_ring) != cudaSuccess)
            return MAC_GATHER;
    }
    std::vector<int> hs(p->n_ring, -1);
    std::vector<double> hS(p->n_ring, 1.0);
    std::vector<long long> ht(p->n_ring, 1);
    for (int j = 0; j < T.A && s - j >= 0; ++j) hs[(s - j) % p->n_ring] = s - j;
    cudaStream_t st = p->stream;
    double ms[MAC_NVAR];
    for (int v = 0; v < MAC_NVAR; ++v) ms[v] = -1.0;
    bool ok = cudaMemcpy(p->d_tune_step, hs.data(), sizeof(int) * p->n_ring, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(p->d_tune_S, hS.data(), sizeof(double) * p->n_ring, cudaMemcpyHostToDevice) == cudaSuccess &&
              cudaMemcpy(p->d_tune_total, ht.data(), sizeof(long long) * p->n_ring, cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return MAC_GATHER;
    }
    TuneFlush fl;
    int best = MAC_GATHER;
    for (int v = 0; v < MAC_NVAR; ++v) {
        if (!mac_built(p, v)) continue;
        ms[v] = tune_time(st, fl, [&] { launch_mac(p, T, s, 0, v, p->d_tune_step, p->d_tune_S, p->d_tune_total, st); });
        count_launch((unsigned long long)(kTuneReps + 1) * mac_kernels(p, v));
        if (ms[v] >= 0 && (ms[v] < ms[best] || ms[best] < 0)) best = v;
    }
    if (cudaGetLastError() != cudaSuccess) return MAC_GATHER;
    std::lock_guard<std::mutex> g(g_tune_mu);
    tune_store(key, best, ms, MAC_NVAR);
    return best;
}

const char* const kFftNames[FFT_NVAR] = {"stages", "lanes", "lanes3", "tma", "tma4", "plane4"};

// One step's FFT passes on the plan's own buffers (forward from the int64
// grid into ring slot 0, inverse from the work spectrum into the grid's
// memory viewed as N^3 floats); the grid is all zero, and the caller clears
// it again afterwards.
void fft_step_passes(lc_plan* p, cudaStream_t st) {
    const long long N = p->N;
    const bool pl = plane_step(p);
    RowR2CArgs r{};
    r.in_mode = ROW_IN_I64;
    r.nrows = N * N;
    r.grid = p->d_grid;
    r.slot_S = p->d_slot_S;
    r.slot_total = p->d_slot_total;
    r.slot = 0;
    r.bf16 = p->history == LC_HISTORY_BF16;
    r.zero_in = N >= 256 ? 1 : 0;
    r.dst = p->d_work;
    r.tw = p->d_tw;
    RowC2RArgs rc{};
    rc.nrows = N * N;
    rc.src = p->d_work;
    rc.out = reinterpret_cast<float*>(p->d_grid);
    rc.scale = 1.0f;
    rc.tw = p->d_tw;
    ColArgs c{};
    c.axis = 0;
    c.dir = -1;
    c.in_mode = COL_IN_PLAIN;
    c.out_mode = COL_OUT_PLAIN;
    c.src = p->d_work;
    c.dst = p->d_work;
    c.tw = p->d_tw;
    if (pl && !p->ops->plane_clustered) {
        // grids with one CTA per plane: only the z + y passes depend on the form
        p->ops->plane_r2c(r, st);
        p->ops->plane_c2r(rc, st);
        count_launch(2);
        return;
    }
    if (pl) {
        p->ops->plane_r2c(r, st);
    } else {
        p->ops->rows_r2c(r, st);
        p->maps.set(c, p->d_err);
        p->ops->cols(c, st);
    }
    c.axis = 1;
    if (p->history == LC_HISTORY_BF16) {
        c.out_mode = COL_OUT_BF16;
        c.dst_bf16 = reinterpret_cast<__nv_bfloat162*>(p->d_ring);
    } else {
        c.out_mode = COL_OUT_RING_F32;
        c.dst = reinterpret_cast<float2*>(p->d_ring);
    }
    c.n_ring = p->n_ring;
    c.wslot = 0;
    p->maps.set(c, p->d_err);
    p->ops->cols(c, st);
    if (pl) {
        p->ops->plane_c2r(rc, st);
        count_launch(3);
        return;
    }
    ColArgs ci{};
    ci.axis = 0;
    ci.dir = 1;
    ci.in_mode = COL_IN_PLAIN;
    ci.out_mode = COL_OUT_PLAIN;
    ci.src = p->d_work;
    ci.dst = p->d_work;
    ci.tw = p->d_tw;
    p->maps.set(ci, p->d_err);
    p->ops->cols(ci, st);
    p->ops->rows_c2r(rc, st);
    count_launch(5);
}

// Pick the FFT pass form for the plan's grid size (plan creation: may
// synchronise).  Forced by lc_fft_set_variant or LC_FFT_VARIANT, else the
// process's earlier choice (or the cache file's), else timed: each form runs
// one step's passes once to warm up, then five times between events; the
// median decides.  The choice holds for every later plan of this size, so
// tables built later all use the same passes.
void choose_fft_variant(lc_plan* p) {
    const FftOps* ops = p->ops;
    const int built = ops->cols_variants();
    if ((built & (built - 1)) == 0) return; // a single form
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto f = g_fft_forced.find(p->N);
        if (f != g_fft_forced.end()) {
            ops->set_cols_variant(f->second);
            return;
        }
    }
    if (const char* f = getenv("LC_FFT_VARIANT")) {
        for (int v = 0; v < FFT_NVAR; ++v)
            if (!strcmp(f, kFftNames[v]) && (built >> v & 1)) {
                ops->set_cols_variant(v);
                return;
            }
    }
    int dev = 0, major = 0, minor = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    char kb[96];
    snprintf(kb, sizeof kb, "fft%dc/sm%d%d/N%d", FFT_NVAR, major, minor, p->N);
    const std::string key(kb);
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        tune_load();
        auto it = g_tune.find(key);
        if (it != g_tune.end() && it->second < FFT_NVAR && (built >> it->second & 1)) {
            ops->set_cols_variant(it->second);
            return;
        }
    }
    cudaStream_t st = p->stream;
    double ms[FFT_NVAR > MAC_NVAR ? FFT_NVAR : MAC_NVAR];
    for (auto& m : ms) m = -1.0;
    int best = ops->cols_variant();
    TuneFlush fl;
    for (int v = 0; v < FFT_NVAR; ++v) {
        if (!(built >> v & 1)) continue;
        ops->set_cols_variant(v);
        ms[v] = tune_time(st, fl, [&] { fft_step_passes(p, st); });
        if (ms[v] >= 0 && (ms[best] < 0 || ms[v] < ms[best])) best = v;
    }
    ops->set_cols_variant(best);
    // the grid's memory held float outputs: clear it for the first deposit
    cudaMemsetAsync(p->d_grid, 0, sizeof(long long) * (size_t)p->N * p->N * p->N, st);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return;
    std::lock_guard<std::mutex> g(g_tune_mu);
    tune_store(key, best, ms, FFT_NVAR);
}

constexpr int kZsTab = 4096; // points of the 1 + z_s(r) table of the sub-cell near field

// room for the near-field source lists of n sources (cells, charges, and the
// sub-cell offsets with near_pm); the old lists are kept on failure
lc_status ensure_near(lc_plan* p, long long n) {
    if (!p->near_on || n <= p->near_cap) return LC_OK;
    long long cap = 1024;
    while (cap < n) cap *= 2;
    long long *cell = nullptr, *q = nullptr;
    double* off = nullptr;
    if (dalloc(p, &cell, (size_t)cap) != cudaSuccess || dalloc(p, &q, (size_t)cap) != cudaSuccess ||
        (p->near_pm && dalloc(p, &off, (size_t)cap * 3) != cudaSuccess)) {
        if (cell) p->bytes -= sizeof(long long) * cap;
        if (q) p->bytes -= sizeof(long long) * cap;
        if (off) p->bytes -= sizeof(double) * 3 * cap;
        cudaFree(cell);
        cudaFree(q);
        cudaFree(off);
        cudaGetLastError();
        return LC_ERR_OOM;
    }
    // graphs captured earlier hold the old lists' addresses: retire, do not free
    for (void* r : {(void*)p->d_src_cell, (void*)p->d_src_q, (void*)p->d_src_off})
        if (r) p->retired.push_back(r);
    p->d_src_cell = cell;
    p->d_src_q = q;
    p->d_src_off = off;
    p->near_cap = cap;
    return LC_OK;
}

size_t table_size(const lc_plan* p, int A) {
    if (A <= 0) return 0;
    return sizeof(float) * (size_t)p->W * ((A + 7) / 8 * 8) + sizeof(double) * A +
           (p->near_on ? sizeof(double) * ((kNearR + 1) * (kNearR + 2) * (kNearR + 3) / 6 + 1) : 0) +
           (p->near_pm ? sizeof(float2) * kZsTab : 0);
}

size_t gsum_size(const lc_plan* p) { return sizeof(float) * 8 * (size_t)p->W + sizeof(double); }

void free_table(lc_plan* p, int s) {
    lc_plan::Table& T = p->tables[s];
    cudaFree(T.ghat);
    cudaFree(T.g0);
    cudaFree(T.gnear);
    cudaFree(T.pmtab);
    if (T.gsum) {
        p->table_bytes -= gsum_size(p);
        p->bytes -= gsum_size(p);
    }
    cudaFree(T.gsum);
    cudaFree(T.g0sum);
    const size_t b = table_size(p, T.A);
    p->table_bytes -= b;
    p->bytes -= b;
    T = lc_plan::Table{};
}

// Make room for a table of `need` bytes for step s under the table budget:
// free unpinned tables of earlier observing steps (oldest first), then of
// later ones (latest first).  The budget is soft: pinned tables stay.
void evict_tables(lc_plan* p, int s, size_t need) {
    if (!p->table_budget) return;
    for (int pass = 0; pass < 2 && p->table_bytes + need > p->table_budget; ++pass) {
        if (pass == 0) {
            for (int v = 0; v < s && p->table_bytes + need > p->table_budget; ++v)
                if (p->tables[v].A > 0 && !p->table_pins[v]) free_table(p, v);
        } else {
            for (int v = p->n_steps - 1; v > s && p->table_bytes + need > p->table_budget; --v)
                if (p->tables[v].A > 0 && !p->table_pins[v]) free_table(p, v);
        }
    }
}

// Build the Ghat table of observing step s (steps 2-3 of Section 2.2).
lc_status build_table(lc_plan* p, int s) {
    lc_plan::Table& T = p->tables[s];
    if (T.A >= 0) return LC_OK;
    StepGeom g = step_geometry(p->cosmo, p->kern, p->z, s, p->l, p->S, true, p->n_shell_max);
    const int A = g.A;
    evict_tables(p, s, table_size(p, A));
    cudaError_t e = cudaSuccess;
    if (A == 0) {
        T.A = 0;
        return LC_OK;
    }
    if (g.ntab > (1LL << 28)) return LC_ERR_UNSUPPORTED_SIZE;
    // host table of g(R), with the s^-3 sample weight folded in
    std::vector<double> gt((size_t)g.ntab);
    g_table(p->cosmo, p->kern, p->z[s + 1], p->l / (2.0 * p->S), g.ntab, gt.data());
    const double inv_s3 = 1.0 / ((double)p->S * p->S * p->S);
    for (auto& v : gt) v *= inv_s3;
    // scratch
    if ((long long)A * p->W > p->gw_cap) {
        cudaFree(p->d_gw);
        p->bytes -= sizeof(double) * p->gw_cap;
        p->gw_cap = 0;
        if ((e = dalloc(p, &p->d_gw, (size_t)A * p->W)) != cudaSuccess) return LC_ERR_OOM;
        p->gw_cap = (long long)A * p->W;
    }
    if (g.ntab > p->gtab_cap) {
        cudaFree(p->d_gtab);
        p->bytes -= sizeof(double) * p->gtab_cap;
        p->gtab_cap = 0;
        if ((e = dalloc(p, &p->d_gtab, (size_t)g.ntab)) != cudaSuccess) return LC_ERR_OOM;
        p->gtab_cap = g.ntab;
    }
    if (!p->d_bnd) {
        const int cap = kMaxShells + 1;
        if (dalloc(p, &p->d_bnd, cap) != cudaSuccess || dalloc(p, &p->d_I, cap) != cudaSuccess ||
            dalloc(p, &p->d_scale, cap) != cudaSuccess)
            return LC_ERR_OOM;
    }
    T.gstride = (A + 7) / 8 * 8;
    if (dalloc(p, &T.ghat, (size_t)p->W * T.gstride) != cudaSuccess) return LC_ERR_OOM;
    if (dalloc(p, &T.g0, (size_t)A) != cudaSuccess ||
        (p->near_on && dalloc(p, &T.gnear, (size_t)(kNearR + 1) * (kNearR + 2) * (kNearR + 3) / 6 + 1) != cudaSuccess) ||
        (p->near_pm && dalloc(p, &T.pmtab, (size_t)kZsTab) != cudaSuccess)) {
        cudaFree(T.gnear);
        T.gnear = nullptr;
        cudaFree(T.ghat);
        cudaFree(T.g0);
        T.ghat = nullptr;
        T.g0 = nullptr;
        return LC_ERR_OOM;
    }
    p->table_bytes += table_size(p, A);
    if (p->near_pm) {
        // the factors of g (Eq. 17) that depend on r only through the
        // light-cone redshift z_s(r), over the innermost shell, for the
        // sub-cell near field: both are smooth in r, so linear interpolation
        // on kZsTab points is far below FP32 rounding
        T.rhi0 = g.hi[0];
        T.rh = g.rh;
        T.rtop = std::min(g.hi[0], g.rh);
        const double zo = p->z[s + 1];
        const double o3 = (1.0 + zo) * (1.0 + zo) * (1.0 + zo) / (16.0 * M_PI * M_PI);
        std::vector<float2> zt(kZsTab);
        for (int k = 0; k < kZsTab; ++k) {
            const double zs = zs_of_r(p->cosmo, zo, T.rtop * k / (kZsTab - 1));
            zt[k].x = (float)(o3 / (1.0 + zs));
            zt[k].y = p->kern.kind == LC_KERNEL_EXP ? 0.0f : (float)(1.0 / (116.29 * alpha_lw(p->cosmo, zs)));
        }
        e = cudaMemcpy(T.pmtab, zt.data(), sizeof(float2) * kZsTab, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(p, e);
    }
    cudaStream_t st = p->stream;
    e = cudaMemcpyAsync(p->d_gtab, gt.data(), sizeof(double) * g.ntab, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->d_bnd, g.bnd.data(), sizeof(long long) * (A + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->d_I, g.I.data(), sizeof(double) * A, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_gw, 0, sizeof(double) * (size_t)A * p->W, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(T.ghat, 0, sizeof(float) * (size_t)p->W * T.gstride, st);
    if (e != cudaSuccess) return cuda_fail(p, e);
    RgfAccumArgs ra;
    ra.N = p->N;
    ra.S = p->S;
    ra.A = A;
    ra.U = (int)ceil(g.rh / p->L) + 1;
    ra.l = p->l;
    ra.W = p->W;
    ra.bnd = p->d_bnd;
    ra.Rh = g.Rh;
    ra.gtab = p->d_gtab;
    ra.gw = p->d_gw;
    ra.rh = g.rh;
    launch_rgf_accum(ra, st);
    launch_rgf_norm(p->N, p->W, A, p->d_gw, p->d_I, p->l * p->l * p->l, p->normalise, p->d_scale, T.g0, st);
    if (p->near_on) launch_near_prep(p->d_gw, p->d_scale, T.gnear, T.g0, st);
    count_launch(2 + (plane_table(p) ? 2ULL : 3ULL) * A + (p->near_on ? 1 : 0));
    for (int j = 0; j < A; ++j) {
        RowR2CArgs r{};
        r.in_mode = ROW_IN_WEDGE;
        r.nrows = (long long)p->N * p->N;
        r.gw = p->d_gw + (size_t)j * p->W;
        r.gscale = p->d_scale + j;
        r.near_r = (p->near_on && j == 0) ? kNearR : -1;
        r.dst = p->d_work;
        r.tw = p->d_tw;
        ColArgs c{};
        c.axis = 0;
        c.dir = -1;
        c.in_mode = COL_IN_PLAIN;
        c.out_mode = COL_OUT_PLAIN;
        c.src = p->d_work;
        c.dst = p->d_work;
        c.tw = p->d_tw;
        if (plane_table(p)) {
            p->ops->plane_r2c(r, st);
        } else {
            p->ops->rows_r2c(r, st);
            p->maps.set(c, p->d_err);
            p->ops->cols(c, st);
        }
        c.axis = 1;
        c.out_mode = COL_OUT_WEDGE;
        c.wedge_out = T.ghat;
        c.wedge_A = T.gstride;
        c.wedge_j = j;
        p->maps.set(c, p->d_err);
        p->ops->cols(c, st);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st); // host table gt must outlive the copy
    if (e != cudaSuccess) return cuda_fail(p, e);
    T.A = A;
    T.mac_variant = choose_mac_variant(p, T, s);
    return LC_OK;
}

lc_status ensure_sources(lc_plan* p, long long n) {
    if (n <= p->src_cap) return LC_OK;
    cudaFree(p->d_pos);
    cudaFree(p->d_lum);
    p->bytes -= sizeof(double) * 4 * p->src_cap;
    p->src_cap = 0;
    long long cap = 1024;
    while (cap < n) cap *= 2;
    if (dalloc(p, &p->d_pos, (size_t)cap * 3) != cudaSuccess || dalloc(p, &p->d_lum, (size_t)cap) != cudaSuccess) {
        cudaFree(p->d_pos);
        cudaFree(p->d_lum);
        p->d_pos = p->d_lum = nullptr;
        return LC_ERR_OOM;
    }
    p->src_cap = cap;
    return LC_OK;
}

bool host_sources_ok(long long n, const double* pos, const double* lum) {
    for (long long i = 0; i < n; ++i) {
        if (!isfinite(lum[i]) || lum[i] < 0.0) return false;
        if (!isfinite(pos[3 * i]) || !isfinite(pos[3 * i + 1]) || !isfinite(pos[3 * i + 2])) return false;
    }
    return true;
}

} // namespace

extern "C" {

lc_status lc_fft_set_variant(int n, int v) {
    const FftOps* ops = ops_for(n);
    if (!ops) return LC_ERR_UNSUPPORTED_SIZE;
    if (v < 0 || v >= FFT_NVAR || !(ops->cols_variants() >> v & 1)) return LC_ERR_UNSUPPORTED_SIZE;
    ops->set_cols_variant(v);
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_fft_forced[n] = v;
    return LC_OK;
}

int lc_fft_variant(int n) {
    const FftOps* ops = ops_for(n);
    return ops ? ops->cols_variant() : -1;
}

const char* lc_status_string(lc_status s) {
    switch (s) {
    case LC_OK: return "ok";
    case LC_ERR_INVALID_ARG: return "invalid argument";
    case LC_ERR_UNSUPPORTED_SIZE: return "unsupported size";
    case LC_ERR_STEP_ORDER: return "step order";
    case LC_ERR_OOM: return "out of device memory";
    case LC_ERR_CUDA: return "CUDA error";
    case LC_ERR_TIMEOUT: return "device wait timed out";
    case LC_ERR_DEVICE_CHECK: return "device-side input check failed";
    }
    return "unknown status";
}

lc_status lc_plan_estimate(int n, const lc_steps* steps, const lc_cosmology* cosmo, size_t* base_bytes,
                           size_t* table_bytes_per_step) {
    if (!ops_for(n) || !valid_steps(steps) || !valid_cosmo(cosmo)) return LC_ERR_INVALID_ARG;
    Cosmo c{cosmo->omega_m, cosmo->h};
    const Kernel k = kernel_of(steps);
    std::vector<double> z;
    if (step_edges(c, k, *steps, z)) return LC_ERR_INVALID_ARG;
    // ring depth from the last step's geometry (the largest horizon)
    int ring = 1;
    for (int s = steps->n_steps - 1; s >= 0 && s >= steps->n_steps - 2; --s) {
        StepGeom g = step_geometry(c, k, z, s, 1.0, 2, false, steps->n_shell_max);
        ring = g.A > ring ? g.A : ring;
    }
    const long long nrp = nrp_of(n), spec = (long long)n * n * nrp, slot = (long long)n * n * (n / 2 + 1);
    const long long hb = steps->history == LC_HISTORY_BF16 ? 4 : 8;
    const long long W = (long long)(n / 2 + 1) * (n / 2 + 2) * (n / 2 + 3) / 6;
    if (base_bytes) *base_bytes = (size_t)(8LL * n * n * n + 8 * spec + hb * slot * ring + 4LL * n * n * n + 4LL * n * n);
    if (table_bytes_per_step) *table_bytes_per_step = (size_t)(4 * W * ring + 8 * ring);
    return LC_OK;
}

lc_status lc_plan_create(int n, double box_mpc, const lc_cosmology* cosmo, const lc_steps* steps, void* cuda_stream,
                         lc_plan** out) {
    if (!out) return LC_ERR_INVALID_ARG;
    *out = nullptr;
    const FftOps* ops = ops_for(n);
    if (!ops) return LC_ERR_UNSUPPORTED_SIZE;
    if (!(box_mpc > 0.0) || !isfinite(box_mpc) || !valid_cosmo(cosmo) || !valid_steps(steps))
        return LC_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return LC_ERR_CUDA;
    }
    lc_plan* p = new (std::nothrow) lc_plan();
    if (!p) return LC_ERR_OOM;
    p->N = n;
    p->L = box_mpc;
    p->l = box_mpc / n;
    p->cosmo = Cosmo{cosmo->omega_m, cosmo->h};
    p->kern = kernel_of(steps);
    p->n_steps = steps->n_steps;
    p->S = steps->subsamples ? steps->subsamples : 4;
    p->history = steps->history;
    p->normalise = steps->normalise ? 1 : 0;
    p->deposit = steps->deposit;
    p->n_shell_max = steps->n_shell_max;
    p->U = steps->out_unit > 0.0 ? steps->out_unit : 1.0;
    p->stream = (cudaStream_t)cuda_stream;
    p->ops = ops;
    p->NRP = nrp_of(n);
    p->spec_elems = (long long)n * n * p->NRP;
    p->W = (long long)(n / 2 + 1) * (n / 2 + 2) * (n / 2 + 3) / 6;
    p->ring_slot = (long long)n * n * (n / 2 + 1);
    if (step_edges(p->cosmo, p->kern, *steps, p->z)) {
        delete p;
        return LC_ERR_INVALID_ARG;
    }
    // active slices per observing step -> ring depth
    p->A_of_step.resize(p->n_steps);
    for (int s = 0; s < p->n_steps; ++s) {
        StepGeom g = step_geometry(p->cosmo, p->kern, p->z, s, p->l, p->S, false, p->n_shell_max);
        if (g.A > kMaxShells) {
            delete p;
            return LC_ERR_UNSUPPORTED_SIZE;
        }
        if (g.ntab > (1LL << 28)) {
            delete p;
            return LC_ERR_UNSUPPORTED_SIZE;
        }
        p->A_of_step[s] = g.A;
        if (g.A > p->n_ring) p->n_ring = g.A;
    }
    p->tables.resize(p->n_steps);
    p->table_pins.assign(p->n_steps, 0);
    cudaError_t e = ensure_init(ops);
    if (e != cudaSuccess) {
        delete p;
        return LC_ERR_CUDA;
    }
    const size_t N3 = (size_t)n * n * n;
    const size_t hb = p->history == LC_HISTORY_BF16 ? 4 : 8;
    bool ok = dalloc(p, &p->d_grid, N3) == cudaSuccess && dalloc(p, &p->d_work, (size_t)p->spec_elems) == cudaSuccess &&
              dalloc(p, (char**)&p->d_ring, hb * (size_t)p->ring_slot * p->n_ring) == cudaSuccess &&
              dalloc(p, &p->d_slot_step, p->n_ring) == cudaSuccess && dalloc(p, &p->d_slot_S, p->n_ring) == cudaSuccess &&
              dalloc(p, &p->d_slot_total, p->n_ring) == cudaSuccess && dalloc(p, &p->d_tw, n) == cudaSuccess &&
              dalloc(p, &p->d_err, 1) == cudaSuccess && dalloc(p, &p->d_maxbits, 1) == cudaSuccess &&
              dalloc(p, &p->d_stamp, 1) == cudaSuccess && dalloc(p, &p->d_rowstamp, (size_t)n * n) == cudaSuccess;
    if (!ok) {
        free_all(p);
        delete p;
        return LC_ERR_OOM;
    }
    p->near_on = steps->near_mode != LC_NEAR_NONE;
    p->near_pm = p->near_on && steps->near_mode == LC_NEAR_SUBCELL;
    if (p->near_on && dalloc(p, &p->d_near, N3) != cudaSuccess) {
        free_all(p);
        delete p;
        return LC_ERR_OOM;
    }
    std::vector<float2> tw = twiddles(n);
    p->maps.make(p->d_work, n);
    e = cudaMemsetAsync(p->d_grid, 0, sizeof(long long) * N3, p->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->d_tw, tw.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, p->stream);
    if (e == cudaSuccess && p->near_on) e = cudaMemsetAsync(p->d_near, 0, sizeof(double) * N3, p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_slot_step, 0xff, sizeof(int) * p->n_ring, p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_slot_total, 0, sizeof(long long) * p->n_ring, p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_slot_S, 0, sizeof(double) * p->n_ring, p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_err, 0, sizeof(int), p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_stamp, 0, sizeof(unsigned), p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_rowstamp, 0, sizeof(unsigned) * (size_t)n * n, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) {
        free_all(p);
        delete p;
        return LC_ERR_CUDA;
    }
    choose_fft_variant(p);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaStreamSynchronize(p->stream)) != cudaSuccess) {
        free_all(p);
        delete p;
        return LC_ERR_CUDA;
    }
    *out = p;
    return LC_OK;
}

lc_status lc_plan_set_table_budget(lc_plan* p, size_t bytes) {
    if (!p) return LC_ERR_INVALID_ARG;
    p->table_budget = bytes;
    return LC_OK;
}

size_t lc_plan_table_bytes(const lc_plan* p) { return p ? p->table_bytes : 0; }

lc_status lc_plan_prepare(lc_plan* p, int b, int e) {
    if (!p) return LC_ERR_INVALID_ARG;
    if (p->failed) return LC_ERR_CUDA;
    if (b < 0 || e > p->n_steps || b > e) return LC_ERR_INVALID_ARG;
    for (int s = b; s < e; ++s) {
        lc_status r = build_table(p, s);
        if (r != LC_OK) return r;
    }
    return LC_OK;
}

// How the deposit grid is cleared between pushes: with a near-field list,
// only the cells the push deposited into (sparse clear); without one, the
// z pass of N >= 256 zeroes what it reads (with row stamps, the stamped rows,
// which hold every non-zero cell), and smaller grids (plane kernels) are
// cleared by a memset before each deposit.
static bool zeroed_by_r2c(const lc_plan* p) { return !p->near_on && p->N >= 256; }
static bool memset_before_deposit(const lc_plan* p) { return !p->near_on && !zeroed_by_r2c(p); }

lc_status lc_push_sources(lc_plan* p, int step, int64_t n_src, const double* pos, const double* lum) {
    if (!p) return LC_ERR_INVALID_ARG;
    if (p->failed) return LC_ERR_CUDA;
    if (step < 0 || step >= p->n_steps || n_src < 0) return LC_ERR_INVALID_ARG;
    if (n_src > 0 && (!pos || !lum)) return LC_ERR_INVALID_ARG;
    if (step <= p->last_pushed) return LC_ERR_STEP_ORDER;
    cudaStream_t st = p->stream;
    const double* dpos = pos;
    const double* dlum = lum;
    cudaError_t e = cudaSuccess;
    if (n_src > 0) {
        const bool dp = is_device_ptr(pos), dl = is_device_ptr(lum);
        if (!dp || !dl) {
            if (!dp && !dl && !host_sources_ok(n_src, pos, lum)) return LC_ERR_INVALID_ARG;
            lc_status r = ensure_sources(p, n_src);
            if (r != LC_OK) return r;
            e = cudaMemcpyAsync(p->d_pos, pos, sizeof(double) * 3 * n_src, dp ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(p->d_lum, lum, sizeof(double) * n_src, dl ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return cuda_fail(p, e);
            dpos = p->d_pos;
            dlum = p->d_lum;
        }
    }
    // the previous push's cells, if no field has cleared them (its list is
    // overwritten by this deposit); inside a capture the graph's launch does it
    if (!p->capturing) clear_grid_cells(p, st);
    if (lc_status r = ensure_near(p, near_entries(p, n_src)); r != LC_OK) return r;
    const int slot = step % p->n_ring;
    // LC_ROW_STAMPS=0: the z pass reads every row of the grid
    static const bool row_stamps = [] {
        const char* v = getenv("LC_ROW_STAMPS");
        return !(v && !strcmp(v, "0"));
    }();
    SlotMeta m{slot, step, p->d_slot_step, p->d_slot_S, p->d_slot_total, row_stamps ? p->d_stamp : nullptr,
               row_stamps ? p->d_rowstamp : nullptr};
    const long long N = p->N;
    {
        Phase ph(p, LC_PHASE_DEPOSIT, n_src > 0 ? 2 : 1);
        if (memset_before_deposit(p)) e = cudaMemsetAsync(p->d_grid, 0, sizeof(long long) * N * N * N, st);
        if (e != cudaSuccess) return cuda_fail(p, e);
        launch_src_prep(dpos, dlum, n_src, p->d_maxbits, p->d_err, m, st);
        if (n_src > 0)
            launch_deposit(dpos, dlum, n_src, p->N, p->l, p->deposit, p->d_maxbits, p->d_grid, m, p->d_err, st,
                           p->near_on ? p->d_src_cell : nullptr, p->near_on ? p->d_src_q : nullptr,
                           p->near_pm ? p->d_src_off : nullptr);
    }
    p->near_n = near_entries(p, n_src);
    if (n_src > 0) p->grid_dirty = true;
    RowR2CArgs r{};
    r.in_mode = ROW_IN_I64;
    r.nrows = N * N;
    r.grid = p->d_grid;
    r.slot_S = p->d_slot_S;
    r.slot_total = p->d_slot_total;
    r.slot = slot;
    r.bf16 = p->history == LC_HISTORY_BF16;
    r.zero_in = zeroed_by_r2c(p) ? 1 : 0;
    r.rowstamp = m.rowstamp;
    r.stamp = m.stamp;
    r.dst = p->d_work;
    r.tw = p->d_tw;
    ColArgs c{};
    c.axis = 0;
    c.dir = -1;
    c.in_mode = COL_IN_PLAIN;
    c.out_mode = COL_OUT_PLAIN;
    c.src = p->d_work;
    c.dst = p->d_work;
    c.tw = p->d_tw;
    if (plane_step(p)) {
        // z and y together, one CTA (or a cluster of four) per x-plane
        Phase ph(p, LC_PHASE_R2C_Z, 1);
        p->ops->plane_r2c(r, st);
    } else {
        {
            Phase ph(p, LC_PHASE_R2C_Z, 1);
            p->ops->rows_r2c(r, st);
        }
        Phase ph(p, LC_PHASE_FWD_Y, 1);
        p->maps.set(c, p->d_err);
        p->ops->cols(c, st);
    }
    c.axis = 1;
    if (p->history == LC_HISTORY_BF16) {
        c.out_mode = COL_OUT_BF16;
        c.dst_bf16 = reinterpret_cast<__nv_bfloat162*>(p->d_ring);
    } else {
        c.out_mode = COL_OUT_RING_F32;
        c.dst = reinterpret_cast<float2*>(p->d_ring);
    }
    c.n_ring = p->n_ring;
    c.wslot = slot;
    // leave the x pass to the field's gather MAC when that field follows in
    // the same capture (grids with plane kernels, whose x pass the fused
    // kernel repeats bit for bit)
    const lc_plan::Table& Tn = p->tables[step];
    if (p->fuse_x && p->capturing && plane_table(p) && Tn.ghat && Tn.A > 0 && Tn.mac_variant == MAC_GATHER) {
        p->x_deferred = slot;
    } else {
        Phase ph(p, LC_PHASE_FWD_X_RING, 1);
        p->maps.set(c, p->d_err);
        p->ops->cols(c, st);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(p, e);
    p->last_pushed = step;
    return LC_OK;
}

static lc_status field_impl(lc_plan* p, int step, float* out, int instant, uint64_t* ticket = nullptr);

lc_status lc_retarded_field(lc_plan* p, int step, float* out) { return field_impl(p, step, out, 0); }

lc_status lc_instant_field(lc_plan* p, int step, float* out) { return field_impl(p, step, out, 1); }

lc_status lc_retarded_field_async(lc_plan* p, int step, float* out, uint64_t* ticket) {
    if (!ticket) return LC_ERR_INVALID_ARG;
    *ticket = 0;
    return field_impl(p, step, out, 0, ticket);
}

lc_status lc_plan_wait(lc_plan* p, uint64_t ticket) {
    if (!p) return LC_ERR_INVALID_ARG;
    if (ticket > p->tickets) return LC_ERR_INVALID_ARG;
    cudaError_t e;
    if (ticket == 0) {
        e = cudaStreamSynchronize(p->stream);
    } else if (ticket <= p->done_upto) {
        return LC_OK;
    } else {
        // the ticket's own event; once kTicketEvents later tickets have been
        // issued it stands for a later copy, which completes after this one
        e = cudaEventSynchronize(p->ev_ticket[(ticket - 1) % lc_plan::kTicketEvents]);
        if (e == cudaSuccess && ticket > p->done_upto) p->done_upto = ticket;
    }
    return e == cudaSuccess ? LC_OK : cuda_fail(p, e);
}

lc_status lc_plan_poll(lc_plan* p, uint64_t ticket, int* done) {
    if (!p || !done) return LC_ERR_INVALID_ARG;
    if (ticket > p->tickets) return LC_ERR_INVALID_ARG;
    *done = 0;
    cudaError_t e;
    if (ticket == 0) e = cudaStreamQuery(p->stream);
    else if (ticket <= p->done_upto) e = cudaSuccess;
    else e = cudaEventQuery(p->ev_ticket[(ticket - 1) % lc_plan::kTicketEvents]);
    if (e == cudaSuccess) {
        if (ticket > p->done_upto) p->done_upto = ticket;
        *done = 1;
        return LC_OK;
    }
    if (e == cudaErrorNotReady) {
        cudaGetLastError();
        return LC_OK;
    }
    return cuda_fail(p, e);
}

// the stage an asynchronous host output computes into: waits (on the plan's
// stream) for the copy that last read it
static cudaError_t async_stage(lc_plan* p, int& k) {
    const long long N3 = p->N * p->N * p->N;
    k = (int)(p->tickets % 2);
    cudaError_t e = cudaSuccess;
    if (!p->copy_stream) e = cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        if (!p->ev_computed[i]) e = cudaEventCreateWithFlags(&p->ev_computed[i], cudaEventDisableTiming);
        if (e == cudaSuccess && !p->ev_copied[i]) e = cudaEventCreateWithFlags(&p->ev_copied[i], cudaEventDisableTiming);
    }
    for (int i = 0; i < lc_plan::kTicketEvents && e == cudaSuccess; ++i)
        if (!p->ev_ticket[i]) e = cudaEventCreateWithFlags(&p->ev_ticket[i], cudaEventDisableTiming);
    if (e == cudaSuccess && !p->d_out_async[k]) e = dalloc(p, &p->d_out_async[k], (size_t)N3);
    if (e == cudaSuccess && p->stage_ticket[k]) e = cudaStreamWaitEvent(p->stream, p->ev_copied[k], 0);
    return e;
}

static lc_status field_impl(lc_plan* p, int step, float* out, int instant, uint64_t* ticket) {
    if (!p || !out) return LC_ERR_INVALID_ARG;
    if (p->failed) return LC_ERR_CUDA;
    if (step < 0 || step >= p->n_steps) return LC_ERR_INVALID_ARG;
    if (step != p->last_pushed) return LC_ERR_STEP_ORDER;
    lc_status rs = build_table(p, step);
    if (rs != LC_OK) return rs;
    cudaStream_t st = p->stream;
    const long long N = p->N, N3 = N * N * N;
    const bool dev_out = is_device_ptr(out);
    const bool async_out = ticket && !dev_out;
    if (async_out && p->capturing) return LC_ERR_INVALID_ARG; // a graph holds device pointers only
    float* dout = out;
    cudaError_t e = cudaSuccess;
    int stage = 0;
    if (async_out) {
        e = async_stage(p, stage);
        if (e == cudaErrorMemoryAllocation) return LC_ERR_OOM;
        if (e != cudaSuccess) return cuda_fail(p, e);
        dout = p->d_out_async[stage];
    } else if (!dev_out) {
        if (!p->d_out_stage && dalloc(p, &p->d_out_stage, (size_t)N3) != cudaSuccess) return LC_ERR_OOM;
        dout = p->d_out_stage;
    }
    lc_plan::Table& T = p->tables[step];
    lc_plan::Table Ti; // the one-shell view of the instantaneous field
    if (instant && T.A > 0) {
        if (!T.gsum) {
            if (p->capturing) return LC_ERR_INVALID_ARG; // built outside a capture only
            if (dalloc(p, &T.gsum, (size_t)8 * p->W) != cudaSuccess) return LC_ERR_OOM;
            if (dalloc(p, &T.g0sum, 1) != cudaSuccess) {
                cudaFree(T.gsum);
                p->bytes -= sizeof(float) * 8 * (size_t)p->W;
                T.gsum = nullptr;
                return LC_ERR_OOM;
            }
            p->table_bytes += gsum_size(p);
            launch_gsum(p->W, T.A, T.gstride, T.ghat, T.g0, T.gsum, T.g0sum, st);
            e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(p, e);
            Ti = T;
            Ti.ghat = T.gsum;
            Ti.g0 = T.g0sum;
            Ti.gstride = 8;
            Ti.A = 1;
            T.inst_variant = choose_mac_variant(p, Ti, step);
        }
        Ti = T;
        Ti.ghat = T.gsum;
        Ti.g0 = T.g0sum;
        Ti.gstride = 8;
        Ti.A = 1;
        Ti.mac_variant = T.inst_variant;
    }
    const lc_plan::Table& M = (instant && T.A > 0) ? Ti : T;
    if (T.A == 0) {
        e = cudaMemsetAsync(dout, 0, sizeof(float) * N3, st);
    } else {
        {
            Phase ph(p, LC_PHASE_MAC_X, mac_kernels(p, M.mac_variant));
            launch_mac(p, M, step, instant, M.mac_variant, p->d_slot_step, p->d_slot_S, p->d_slot_total, st);
        }
        ColArgs c{};
        c.dir = 1;
        c.out_mode = COL_OUT_PLAIN;
        c.dst = p->d_work;
        c.tw = p->d_tw;
        c.axis = 0;
        c.in_mode = COL_IN_PLAIN;
        c.src = p->d_work;
        RowC2RArgs r{};
        r.nrows = N * N;
        r.src = p->d_work;
        r.out = dout;
        r.scale = (float)(p->U / (double)N3);
        r.tw = p->d_tw;
        const int nslot = step % p->n_ring;
        const bool near_list = p->near_on && p->near_n > 0 && !p->near_pm;
        NearScatter ns{p->d_src_cell, p->d_src_q, p->near_n, T.gnear, p->d_slot_S, nslot, p->U, p->d_near, 0};
        bool near_done = false;
        if (plane_step(p)) {
            // y and z together, one CTA (or a cluster of four) per x-plane; a
            // short near-field list runs on extra CTAs of the same launch, on
            // the SMs that the planes leave idle, instead of a launch of its own.
            // LC_NEAR_CTAS=0: always the separate launch
            static const bool fuse_near = [] {
                const char* v = getenv("LC_NEAR_CTAS");
                return !(v && !strcmp(v, "0"));
            }();
            if (near_list && fuse_near) {
                const int c = p->ops->plane_near_ctas(p->near_n * kNearCube, sm_count());
                if (c > 0) {
                    r.near = ns;
                    r.near.ctas = c;
                    near_done = true;
                }
            }
            Phase ph(p, LC_PHASE_C2R_Z, 1);
            p->ops->plane_c2r(r, st);
        } else {
            {
                Phase ph(p, LC_PHASE_INV_Y, 1);
                p->maps.set(c, p->d_err);
                p->ops->cols(c, st);
            }
            Phase ph(p, LC_PHASE_C2R_Z, 1);
            p->ops->rows_c2r(r, st);
        }
        if (p->near_on && p->near_n > 0) {
            // innermost shell's near cube, summed exactly in FP64 and folded in
            Phase ph(p, LC_PHASE_NEAR, near_done ? 1 : 2);
            if (p->near_pm) {
                NearPmArgs na{};
                na.cell = p->d_src_cell;
                na.q = p->d_src_q;
                na.off = p->d_src_off;
                na.n = p->near_n;
                na.N = p->N;
                na.S = p->S;
                na.l = p->l;
                na.L = p->L;
                na.rtop = T.rtop;
                na.rhi = T.rhi0;
                na.rh = T.rh;
                na.rtop2f = (float)(T.rtop * T.rtop);
                na.win2f = (float)(1e-5 * (T.rtop * T.rtop + T.rtop * p->l));
                {
                    const double reach = T.rtop + 0.5 * 1.7320508075688772 * p->l;
                    na.prune2f = (float)(reach * reach * (1.0 + 1e-5));
                }
                na.U = (int)ceil((T.rtop + 2.0 * (kNearR + 1) * p->l) / p->L) + 1;
                na.tab = T.pmtab;
                na.K = kZsTab;
                na.kind = p->kern.kind;
                // Eq. 15's cut as r / (116.29 alpha); none with the rough horizon
                // (the rough horizon is rtop's bound, f_mod clamped at 0)
                na.xcut = p->kern.kind == kKernelLwRough ? 3.0e38f : (float)(97.39 / 116.29);
                na.inv_klen = (float)(1.0 / p->kern.length);
                na.kmax = (float)p->kern.rmax;
                na.f0 = T.gnear + (kNearR + 1) * (kNearR + 2) * (kNearR + 3) / 6;
                na.slot_S = p->d_slot_S;
                na.slot = nslot;
                na.U_out = p->U;
                launch_near_pm(na, p->d_near, st);
            } else if (!near_done) {
                launch_near_scatter(ns, p->N, st);
            }
            launch_near_fold(p->d_src_cell, p->d_src_q, p->near_n, p->N, p->d_near, dout, p->d_grid, st);
            p->grid_dirty = false; // the fold cleared the deposit cells
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && p->grid_dirty && p->near_on) {
        // no fold ran (no active shell, or no sources): clear the cells here
        clear_grid_cells(p, st);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && async_out) {
        // copy out on the copy stream once computed; the next step's kernels
        // run meanwhile on the plan's stream
        e = cudaEventRecord(p->ev_computed[stage], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->copy_stream, p->ev_computed[stage], 0);
        // page-locked and 16-byte aligned: a kernel on the copy stream writes
        // it through the buffer's device view (SM stores over the host link;
        // with several plans serving at once this kept up better than the
        // copy engines), with a small grid so that the copy holds few SM
        // slots: serving c5 end to end, 231 fields/s by the copy engine,
        // 340 with 152 CTAs, 386 with 24, 409 with 16, 419 with 12, and
        // 402-439 (the spread between runs) with 4 to 8.  LC_D2H=ce: always
        // the copy engine.  LC_D2H_CTAS: the copy kernel's CTAs (default 8).
        static const bool sm_copy = [] {
            const char* v = getenv("LC_D2H");
            return !(v && !strcmp(v, "ce"));
        }();
        static const int copy_ctas = [] {
            const char* v = getenv("LC_D2H_CTAS");
            const int c = v ? atoi(v) : 0;
            return c > 0 ? c : 8;
        }();
        void* hv = sm_copy ? pinned_device_view(out) : nullptr;
        if (e == cudaSuccess && hv && (reinterpret_cast<uintptr_t>(hv) & 15) == 0) {
            launch_copy_out(N3 / 4, reinterpret_cast<const float4*>(dout), reinterpret_cast<float4*>(hv),
                            copy_ctas, p->copy_stream);
            count_launch(1);
            e = cudaGetLastError();
        } else if (e == cudaSuccess) {
            e = cudaMemcpyAsync(out, dout, sizeof(float) * N3, cudaMemcpyDeviceToHost, p->copy_stream);
        }
        if (e == cudaSuccess) e = cudaEventRecord(p->ev_copied[stage], p->copy_stream);
        if (e == cudaSuccess)
            e = cudaEventRecord(p->ev_ticket[p->tickets % lc_plan::kTicketEvents], p->copy_stream);
        if (e == cudaSuccess) {
            *ticket = ++p->tickets;
            p->stage_ticket[stage] = *ticket;
        }
    } else if (e == cudaSuccess && !dev_out) {
        // page-locked and 16-byte aligned: the SMs write it through its device
        // view (faster than one copy-engine transfer); otherwise a copy
        void* hv = pinned_device_view(out);
        if (hv && (reinterpret_cast<uintptr_t>(hv) & 15) == 0) {
            launch_copy_out(N3 / 4, reinterpret_cast<const float4*>(dout), reinterpret_cast<float4*>(hv), 4 * sm_count(),
                            st);
            count_launch(1);
            e = cudaGetLastError();
        } else {
            e = cudaMemcpyAsync(out, dout, sizeof(float) * N3, cudaMemcpyDeviceToHost, st);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    return cuda_fail(p, e);
}

lc_status lc_plan_reset(lc_plan* p) {
    if (!p) return LC_ERR_INVALID_ARG;
    if (p->failed) return LC_ERR_CUDA;
    cudaError_t e = cudaMemsetAsync(p->d_slot_step, 0xff, sizeof(int) * p->n_ring, p->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_slot_total, 0, sizeof(long long) * p->n_ring, p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e);
    p->last_pushed = -1;
    return LC_OK;
}

// ---------------------------------------------------------------- checkpoint
namespace {
constexpr unsigned long long kCkptMagic = 0x31304b43505443ULL; // "CTPCK01"
struct CkptHeader {
    unsigned long long magic;
    int version, N, n_steps, n_ring, history, last_pushed;
    long long near_n;
    unsigned long long params_hash;
    long long ring_bytes;
    unsigned char pad[256 - 8 - 6 * 4 - 8 - 8 - 8];
};
static_assert(sizeof(CkptHeader) == 256, "checkpoint header is 256 bytes");

// FNV-1a over the bytes of every method parameter
unsigned long long params_hash(const lc_plan* p) {
    unsigned long long h = 1469598103934665603ULL;
    auto mix = [&h](const void* d, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(d);
        for (size_t i = 0; i < n; ++i) {
            h ^= b[i];
            h *= 1099511628211ULL;
        }
    };
    mix(&p->N, sizeof p->N);
    mix(&p->L, sizeof p->L);
    mix(&p->cosmo, sizeof p->cosmo);
    mix(&p->n_steps, sizeof p->n_steps);
    mix(&p->S, sizeof p->S);
    mix(&p->history, sizeof p->history);
    mix(&p->normalise, sizeof p->normalise);
    mix(&p->U, sizeof p->U);
    mix(p->z.data(), sizeof(double) * p->z.size());
    mix(&p->kern.kind, sizeof p->kern.kind);
    mix(&p->kern.length, sizeof p->kern.length);
    mix(&p->kern.rmax, sizeof p->kern.rmax);
    mix(&p->near_pm, sizeof p->near_pm);
    mix(&p->deposit, sizeof p->deposit);
    mix(&p->n_shell_max, sizeof p->n_shell_max);
    return h;
}

size_t ring_bytes_of(const lc_plan* p) {
    return (size_t)p->n_ring * p->ring_slot * (p->history == LC_HISTORY_BF16 ? 4 : 8);
}

size_t meta_bytes_of(const lc_plan* p, long long near_n) {
    return (size_t)p->n_ring * (sizeof(int) + sizeof(double) + sizeof(long long)) +
           (size_t)near_n * 2 * sizeof(long long) + (p->near_pm ? (size_t)near_n * 3 * sizeof(double) : 0);
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }
} // namespace

size_t lc_plan_checkpoint_bytes(const lc_plan* p) {
    if (!p) return 0;
    return sizeof(CkptHeader) + align256(meta_bytes_of(p, p->near_n)) + ring_bytes_of(p);
}

lc_status lc_plan_save(lc_plan* p, void* buf, size_t size) {
    if (!p || !buf) return LC_ERR_INVALID_ARG;
    if (p->failed) return LC_ERR_CUDA;
    if (size < lc_plan_checkpoint_bytes(p)) return LC_ERR_INVALID_ARG;
    CkptHeader h{};
    h.magic = kCkptMagic;
    h.version = 1;
    h.N = p->N;
    h.n_steps = p->n_steps;
    h.n_ring = p->n_ring;
    h.history = p->history;
    h.last_pushed = p->last_pushed;
    h.near_n = p->near_n;
    h.params_hash = params_hash(p);
    h.ring_bytes = (long long)ring_bytes_of(p);
    unsigned char* b = static_cast<unsigned char*>(buf);
    cudaStream_t st = p->stream;
    const size_t nr = (size_t)p->n_ring;
    size_t off = sizeof h;
    cudaError_t e = cudaMemcpyAsync(b, &h, sizeof h, cudaMemcpyDefault, st);
    auto put = [&](const void* src, size_t n) {
        if (e == cudaSuccess && n) e = cudaMemcpyAsync(b + off, src, n, cudaMemcpyDefault, st);
        off += n;
    };
    put(p->d_slot_step, nr * sizeof(int));
    put(p->d_slot_S, nr * sizeof(double));
    put(p->d_slot_total, nr * sizeof(long long));
    put(p->d_src_cell, (size_t)p->near_n * sizeof(long long));
    put(p->d_src_q, (size_t)p->near_n * sizeof(long long));
    if (p->near_pm) put(p->d_src_off, (size_t)p->near_n * 3 * sizeof(double));
    off = sizeof h + align256(meta_bytes_of(p, p->near_n));
    put(p->d_ring, ring_bytes_of(p));
    if (e == cudaSuccess) e = cudaStreamSynchronize(st); // the header copy reads a stack object
    if (e != cudaSuccess) return cuda_fail(p, e);
    return LC_OK;
}

lc_status lc_plan_load(lc_plan* p, const void* buf, size_t size) {
    if (!p || !buf) return LC_ERR_INVALID_ARG;
    if (p->failed) return LC_ERR_CUDA;
    if (size < sizeof(CkptHeader)) return LC_ERR_INVALID_ARG;
    CkptHeader h{};
    cudaStream_t st = p->stream;
    cudaError_t e = cudaMemcpyAsync(&h, buf, sizeof h, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(p, e);
    if (h.magic != kCkptMagic || h.version != 1 || h.N != p->N || h.n_steps != p->n_steps ||
        h.n_ring != p->n_ring || h.history != p->history || h.params_hash != params_hash(p) ||
        h.ring_bytes != (long long)ring_bytes_of(p) || h.last_pushed < -1 || h.last_pushed >= p->n_steps ||
        h.near_n < 0 || (!p->near_on && h.near_n != 0))
        return LC_ERR_INVALID_ARG;
    if (size < sizeof h + align256(meta_bytes_of(p, h.near_n)) + ring_bytes_of(p)) return LC_ERR_INVALID_ARG;
    clear_grid_cells(p, st); // the current list's cells, before the list is replaced
    if (lc_status r = ensure_near(p, h.near_n); r != LC_OK) return r;
    const unsigned char* b = static_cast<const unsigned char*>(buf);
    const size_t nr = (size_t)p->n_ring;
    size_t off = sizeof h;
    auto get = [&](void* dst, size_t n) {
        if (e == cudaSuccess && n) e = cudaMemcpyAsync(dst, b + off, n, cudaMemcpyDefault, st);
        off += n;
    };
    get(p->d_slot_step, nr * sizeof(int));
    get(p->d_slot_S, nr * sizeof(double));
    get(p->d_slot_total, nr * sizeof(long long));
    get(p->d_src_cell, (size_t)h.near_n * sizeof(long long));
    get(p->d_src_q, (size_t)h.near_n * sizeof(long long));
    if (p->near_pm) get(p->d_src_off, (size_t)h.near_n * 3 * sizeof(double));
    off = sizeof h + align256(meta_bytes_of(p, h.near_n));
    get(p->d_ring, ring_bytes_of(p));
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(p, e);
    p->last_pushed = h.last_pushed;
    p->near_n = h.near_n;
    return LC_OK;
}

lc_status lc_plan_check(lc_plan* p) {
    if (!p) return LC_ERR_INVALID_ARG;
    if (p->failed) return LC_ERR_CUDA;
    int err = 0;
    cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e == cudaSuccess) e = cudaMemcpy(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(p, e);
    if (err) {
        cudaMemset(p->d_err, 0, sizeof(int));
        return LC_ERR_DEVICE_CHECK;
    }
    return LC_OK;
}

lc_status lc_plan_set_stream(lc_plan* p, void* s) {
    if (!p) return LC_ERR_INVALID_ARG;
    p->stream = (cudaStream_t)s;
    return LC_OK;
}

lc_status lc_plan_destroy(lc_plan* p) {
    if (!p) return LC_ERR_INVALID_ARG;
    cudaStreamSynchronize(p->stream);
    cudaGetLastError();
    free_all(p);
    delete p;
    return LC_OK;
}

size_t lc_plan_device_bytes(const lc_plan* p) { return p ? p->bytes : 0; }

lc_status lc_plan_set_timing(lc_plan* p, int enable) {
    if (!p) return LC_ERR_INVALID_ARG;
    p->timing = enable != 0;
    return LC_OK;
}

lc_status lc_plan_timing(lc_plan* p, double* ms, int64_t* launches, int reset) {
    if (!p) return LC_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e);
    for (auto& m : p->marks) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, m.a, m.b) == cudaSuccess) p->ms[m.phase] += t;
        else cudaGetLastError();
        p->pool.push_back(m.a);
        p->pool.push_back(m.b);
    }
    p->marks.clear();
    for (auto* g : p->graphs) harvest_graph(p, g);
    for (int i = 0; i < LC_N_PHASES; ++i) {
        if (ms) ms[i] = p->ms[i];
        if (launches) launches[i] = p->launches[i];
        if (reset) {
            p->ms[i] = 0;
            p->launches[i] = 0;
        }
    }
    return LC_OK;
}

uint64_t lc_kernel_launches(void) { return g_launches.load(); }

lc_status lc_step_shells(const lc_plan* p, int step, int* n_active, double* r_lo, double* r_hi, double* r_h,
                         double* shell_integral) {
    if (!p || step < 0 || step >= p->n_steps) return LC_ERR_INVALID_ARG;
    StepGeom g = step_geometry(p->cosmo, p->kern, p->z, step, p->l, p->S, shell_integral != nullptr, p->n_shell_max);
    if (n_active) *n_active = g.A;
    for (int j = 0; j < g.A; ++j) {
        if (r_lo) r_lo[j] = g.lo[j];
        if (r_hi) r_hi[j] = g.hi[j];
        if (shell_integral) shell_integral[j] = g.I[j];
    }
    if (r_h) *r_h = g.rh;
    return LC_OK;
}

lc_status lc_plan_info(const lc_plan* p, lc_plan_info_t* info) {
    if (!p || !info) return LC_ERR_INVALID_ARG;
    info->n = p->N;
    info->n_steps = p->n_steps;
    info->n_ring = p->n_ring;
    info->history = p->history;
    info->wedge_size = (int)p->W;
    info->spectrum_row = p->NRP;
    info->box_mpc = p->L;
    info->z_edges = p->z.data();
    return LC_OK;
}

int lc_autotune_report(char* buf, int size) {
    std::lock_guard<std::mutex> g(g_tune_mu);
    tune_load();
    std::string out;
    for (auto& kv : g_tune)
        out += kv.first + " " +
               (kv.first.compare(0, 3, "fft") == 0 ? (kv.second < FFT_NVAR ? kFftNames[kv.second] : "?")
                                                   : (kv.second < MAC_NVAR ? kMacNames[kv.second] : "?")) +
               "\n";
    if (buf && size > 0) {
        const int n = (int)out.size() < size - 1 ? (int)out.size() : size - 1;
        memcpy(buf, out.data(), n);
        buf[n] = 0;
    }
    return (int)out.size();
}

lc_status lc_plan_green_wedge(lc_plan* p, int step, int lookback, float* out, double* ghat0) {
    if (!p || !out || step < 0 || step >= p->n_steps) return LC_ERR_INVALID_ARG;
    if (p->failed) return LC_ERR_CUDA;
    lc_status r = build_table(p, step);
    if (r != LC_OK) return r;
    const lc_plan::Table& T = p->tables[step];
    if (lookback < 0 || lookback >= T.A) return LC_ERR_INVALID_ARG;
    // strided column j of the [W][A] table
    std::vector<float> col((size_t)p->W);
    double g0 = 0.0;
    cudaError_t e = cudaMemcpy2DAsync(col.data(), sizeof(float), T.ghat + lookback, sizeof(float) * T.gstride,
                                      sizeof(float), (size_t)p->W, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&g0, T.g0 + lookback, sizeof(double), cudaMemcpyDeviceToHost, p->stream);
    const int Wn = (kNearR + 1) * (kNearR + 2) * (kNearR + 3) / 6;
    std::vector<double> gn(Wn, 0.0);
    const bool add_near = p->near_on && lookback == 0;
    if (e == cudaSuccess && add_near)
        e = cudaMemcpyAsync(gn.data(), T.gnear, sizeof(double) * Wn, cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e);
    if (add_near) {
        // the FFT path holds shell 0 without its near cube: add the cube's
        // (real, even) transform back so that the full Ghat_0 is returned
        const int N = p->N, M = N / 2, R = kNearR;
        std::vector<double> cs(N);
        for (int m = 0; m < N; ++m) cs[m] = cos(2.0 * 3.141592653589793238462643383279502884 * m / N);
        auto wi = [](int a, int b, int c) {
            int t;
            if (a > b) { t = a; a = b; b = t; }
            if (b > c) { t = b; b = c; c = t; }
            if (a > b) { t = a; a = b; b = t; }
            return (long long)c * (c + 1) * (c + 2) / 6 + (long long)b * (b + 1) / 2 + a;
        };
        double cube = 0.0;
        for (int dx = -R; dx <= R; ++dx)
            for (int dy = -R; dy <= R; ++dy)
                for (int dz = -R; dz <= R; ++dz) cube += gn[wi(abs(dx), abs(dy), abs(dz))];
        long long w = 0;
        for (int c = 0; c <= M; ++c)
            for (int b = 0; b <= c; ++b)
                for (int a = 0; a <= b; ++a, ++w) {
                    double v = 0.0;
                    for (int dx = -R; dx <= R; ++dx)
                        for (int dy = -R; dy <= R; ++dy)
                            for (int dz = -R; dz <= R; ++dz) {
                                const long long ph = ((long long)a * dx + (long long)b * dy + (long long)c * dz) % N;
                                v += gn[wi(abs(dx), abs(dy), abs(dz))] * cs[(ph + N) % N];
                            }
                    col[w] = (float)((double)col[w] + v);
                }
        g0 += cube;
    }
    e = cudaMemcpy(out, col.data(), sizeof(float) * p->W, cudaMemcpyDefault);
    if (e != cudaSuccess) return cuda_fail(p, e);
    if (ghat0) *ghat0 = g0;
    return LC_OK;
}

// ------------------------------------------------------------ step graphs
// Checks and preparation shared by the graph captures: device pointers
// only, the step's table built and every buffer the step needs allocated
// (nothing may be allocated or synchronised during a capture).
static lc_status prepare_capture(lc_plan* p, int step, int64_t n_src, const double* pos, const double* lum,
                                 float* out) {
    if (!p || !out) return LC_ERR_INVALID_ARG;
    if (p->failed) return LC_ERR_CUDA;
    if (step < 0 || step >= p->n_steps || n_src < 0) return LC_ERR_INVALID_ARG;
    if (!is_device_ptr(out) || (n_src > 0 && (!pos || !lum || !is_device_ptr(pos) || !is_device_ptr(lum))))
        return LC_ERR_INVALID_ARG; // a graph holds device pointers only
    lc_status r = build_table(p, step);
    if (r != LC_OK) return r;
    if (lc_status r2 = ensure_near(p, near_entries(p, n_src)); r2 != LC_OK) return r2;
    return LC_OK;
}

lc_status lc_graph_create(lc_plan* p, int step, int64_t n_src, const double* pos, const double* lum, float* out,
                          lc_step_graph** out_graph) {
    if (!out_graph) return LC_ERR_INVALID_ARG;
    *out_graph = nullptr;
    lc_status r = prepare_capture(p, step, n_src, pos, lum, out);
    if (r != LC_OK) return r;
    lc_step_graph* g = new (std::nothrow) lc_step_graph();
    if (!g) return LC_ERR_OOM;
    g->p = p;
    g->step = step;
    ++p->table_pins[step]; // the graph holds the table's address
    g->n_src = n_src;
    cudaStream_t cap_stream = nullptr, user_stream = p->stream;
    cudaError_t e = cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete g;
        return cuda_fail(p, e);
    }
    const int saved_last = p->last_pushed;
    const long long saved_near = p->near_n;
    const bool saved_dirty = p->grid_dirty;
    const size_t marks0 = p->marks.size();
    for (int i = 0; i < LC_N_PHASES; ++i) p->cap_kernels[i] = 0;
    p->stream = cap_stream;
    p->capturing = true;
    p->last_pushed = step - 1;
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal);
    lc_status rs = LC_OK;
    if (e == cudaSuccess) {
        p->fuse_x = true;
        rs = lc_push_sources(p, step, n_src, pos, lum);
        if (rs == LC_OK) rs = lc_retarded_field(p, step, out);
        p->fuse_x = false;
        if (rs == LC_OK && p->x_deferred >= 0) rs = LC_ERR_INVALID_ARG; // the field did not take the x pass
        p->x_deferred = -1;
        cudaError_t e2 = cudaStreamEndCapture(cap_stream, &graph);
        if (e == cudaSuccess) e = e2;
    }
    p->capturing = false;
    p->stream = user_stream;
    p->last_pushed = saved_last;
    p->near_n = saved_near;
    p->grid_dirty = saved_dirty;
    g->marks.assign(p->marks.begin() + marks0, p->marks.end());
    p->marks.resize(marks0);
    for (int i = 0; i < LC_N_PHASES; ++i) g->kernels[i] = p->cap_kernels[i];
    if (e == cudaSuccess && rs == LC_OK) e = cudaGraphInstantiate(&g->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap_stream);
    if (rs != LC_OK || e != cudaSuccess) {
        for (auto& m : g->marks) {
            p->pool.push_back(m.a);
            p->pool.push_back(m.b);
        }
        delete g;
        cudaGetLastError();
        if (rs != LC_OK) return rs;
        return LC_ERR_CUDA; // capture failed: the plan itself is still usable
    }
    p->graphs.push_back(g);
    *out_graph = g;
    return LC_OK;
}

lc_status lc_graph_launch(lc_step_graph* g) {
    if (!g || !g->p) return LC_ERR_INVALID_ARG;
    lc_plan* p = g->p;
    if (p->failed) return LC_ERR_CUDA;
    if (g->step <= p->last_pushed) return LC_ERR_STEP_ORDER;
    harvest_graph(p, g); // its previous replay, long finished in a step cycle
    clear_grid_cells(p, p->stream); // a push outside the graph left its cells (the graph's field clears its own)
    cudaError_t e = cudaGraphLaunch(g->exec, p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e);
    p->grid_dirty = false;
    p->last_pushed = g->step;
    p->near_n = near_entries(p, g->n_src);
    long long tot = 0;
    for (int i = 0; i < LC_N_PHASES; ++i) {
        p->launches[i] += g->kernels[i];
        tot += g->kernels[i];
    }
    count_launch((unsigned long long)tot);
    g->pending = true;
    return LC_OK;
}

lc_status lc_graph_destroy(lc_step_graph* g) {
    if (!g || !g->p) return LC_ERR_INVALID_ARG;
    lc_plan* p = g->p;
    cudaStreamSynchronize(p->stream);
    harvest_graph(p, g);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    for (auto& m : g->marks) {
        p->pool.push_back(m.a);
        p->pool.push_back(m.b);
    }
    for (size_t i = 0; i < p->graphs.size(); ++i)
        if (p->graphs[i] == g) {
            p->graphs.erase(p->graphs.begin() + i);
            break;
        }
    --p->table_pins[g->step];
    delete g;
    return LC_OK;
}

// ------------------------------------------------------------ batched instances
lc_status lc_batch_graph_create(lc_plan* const* plans, int n, const int* steps, const int64_t* n_src,
                                const double* const* pos, const double* const* lum, float* const* outs,
                                lc_batch_graph** out_graph) {
    if (!plans || n < 1 || !steps || !n_src || !outs || !out_graph) return LC_ERR_INVALID_ARG;
    *out_graph = nullptr;
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < i; ++k)
            if (plans[i] == plans[k]) return LC_ERR_INVALID_ARG; // one step per plan per batch
    for (int i = 0; i < n; ++i) {
        lc_status r = prepare_capture(plans[i], steps[i], n_src[i], pos ? pos[i] : nullptr, lum ? lum[i] : nullptr,
                                      outs[i]);
        if (r != LC_OK) return r;
    }
    // a batch graph may outlive the bookkeeping of its plans, so the tables it
    // captured stay pinned for the lives of those plans
    for (int i = 0; i < n; ++i) ++plans[i]->table_pins[steps[i]];
    lc_batch_graph* g = new (std::nothrow) lc_batch_graph();
    if (!g) return LC_ERR_OOM;
    g->plans.assign(plans, plans + n);
    g->steps.assign(steps, steps + n);
    g->n_src.assign(n_src, n_src + n);
    // origin stream s0 forks one branch per instance (its own stream) and joins them
    cudaStream_t s0 = nullptr;
    std::vector<cudaStream_t> br(n, nullptr);
    std::vector<cudaEvent_t> done(n, nullptr);
    cudaEvent_t fork = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s0, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&br[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done[i], cudaEventDisableTiming);
    }
    cudaGraph_t graph = nullptr;
    lc_status rs = LC_OK;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaEventRecord(fork, s0);
        for (int i = 0; i < n && rs == LC_OK; ++i) {
            lc_plan* p = plans[i];
            cudaStreamWaitEvent(br[i], fork, 0);
            const cudaStream_t user_stream = p->stream;
            const int saved_last = p->last_pushed;
            const long long saved_near = p->near_n;
            const bool saved_dirty = p->grid_dirty;
            const bool saved_timing = p->timing;
            for (int k = 0; k < LC_N_PHASES; ++k) p->cap_kernels[k] = 0;
            p->stream = br[i];
            p->capturing = true;
            p->timing = false;
            p->last_pushed = steps[i] - 1;
            rs = lc_push_sources(p, steps[i], n_src[i], pos ? pos[i] : nullptr, lum ? lum[i] : nullptr);
            if (rs == LC_OK) rs = lc_retarded_field(p, steps[i], outs[i]);
            for (int k = 0; k < LC_N_PHASES; ++k) g->kernels += p->cap_kernels[k];
            p->capturing = false;
            p->timing = saved_timing;
            p->stream = user_stream;
            p->last_pushed = saved_last;
            p->near_n = saved_near;
            p->grid_dirty = saved_dirty;
            cudaEventRecord(done[i], br[i]);
            cudaStreamWaitEvent(s0, done[i], 0);
        }
        cudaError_t e2 = cudaStreamEndCapture(s0, &graph);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess && rs == LC_OK) e = cudaGraphInstantiate(&g->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    for (int i = 0; i < n; ++i) {
        if (br[i]) cudaStreamDestroy(br[i]);
        if (done[i]) cudaEventDestroy(done[i]);
    }
    if (fork) cudaEventDestroy(fork);
    if (s0) cudaStreamDestroy(s0);
    if (rs != LC_OK || e != cudaSuccess) {
        delete g;
        cudaGetLastError();
        return rs != LC_OK ? rs : LC_ERR_CUDA;
    }
    *out_graph = g;
    return LC_OK;
}

lc_status lc_batch_graph_launch(lc_batch_graph* g, void* stream) {
    if (!g || !g->exec) return LC_ERR_INVALID_ARG;
    for (size_t i = 0; i < g->plans.size(); ++i) {
        if (g->plans[i]->failed) return LC_ERR_CUDA;
        if (g->steps[i] <= g->plans[i]->last_pushed) return LC_ERR_STEP_ORDER;
    }
    for (auto* p : g->plans) clear_grid_cells(p, (cudaStream_t)stream);
    cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        for (auto* p : g->plans) p->failed = true;
        return LC_ERR_CUDA;
    }
    for (size_t i = 0; i < g->plans.size(); ++i) {
        g->plans[i]->grid_dirty = false;
        g->plans[i]->last_pushed = g->steps[i];
        g->plans[i]->near_n = near_entries(g->plans[i], g->n_src[i]);
    }
    count_launch((unsigned long long)g->kernels);
    return LC_OK;
}

lc_status lc_batch_graph_destroy(lc_batch_graph* g) {
    if (!g) return LC_ERR_INVALID_ARG;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    delete g;
    return LC_OK;
}

// ------------------------------------------------------------ stand-alone kernels
lc_status lc_fdiff_map(int64_t n, const float* j_retarded, const float* j_instant, float* out, void* stream) {
    if (n < 0 || (n > 0 && (!j_retarded || !j_instant || !out))) return LC_ERR_INVALID_ARG;
    if (n > 0 && (!is_device_ptr(j_retarded) || !is_device_ptr(j_instant) || !is_device_ptr(out)))
        return LC_ERR_INVALID_ARG;
    launch_fdiff(n, j_retarded, j_instant, out, (cudaStream_t)stream);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) count_launch(n > 0 ? 1 : 0);
    return e == cudaSuccess ? LC_OK : LC_ERR_CUDA;
}

lc_status lc_deposit_grid(int n, double box, int deposit, int64_t n_src, const double* pos, const double* lum,
                          int64_t* grid, double* scale, int64_t* total, void* stream) {
    if (n < 1 || n > 4096 || !(box > 0.0) || n_src < 0 || !grid || (n_src > 0 && (!pos || !lum)))
        return LC_ERR_INVALID_ARG;
    if (deposit != LC_DEPOSIT_NGP && deposit != LC_DEPOSIT_CIC) return LC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    lc_plan tmp; // only for the allocation helper
    const size_t N3 = (size_t)n * n * n;
    double *dpos = nullptr, *dlum = nullptr, *dS = nullptr;
    long long *dgrid = nullptr, *dtot = nullptr;
    int *dstep = nullptr, *derr = nullptr;
    unsigned long long* dmax = nullptr;
    const bool pos_dev = n_src > 0 && is_device_ptr(pos), lum_dev = n_src > 0 && is_device_ptr(lum),
               grid_dev = is_device_ptr(grid);
    if (n_src > 0 && !pos_dev && !lum_dev && !host_sources_ok(n_src, pos, lum)) return LC_ERR_INVALID_ARG;
    cudaError_t e = cudaSuccess;
    auto cleanup = [&]() {
        if (!pos_dev) cudaFree(dpos);
        if (!lum_dev) cudaFree(dlum);
        if (!grid_dev) cudaFree(dgrid);
        cudaFree(dS);
        cudaFree(dtot);
        cudaFree(dstep);
        cudaFree(derr);
        cudaFree(dmax);
    };
    bool ok = true;
    if (pos_dev) dpos = const_cast<double*>(pos);
    else ok = ok && dalloc(&tmp, &dpos, (size_t)3 * n_src) == cudaSuccess;
    if (lum_dev) dlum = const_cast<double*>(lum);
    else ok = ok && dalloc(&tmp, &dlum, (size_t)n_src) == cudaSuccess;
    if (grid_dev) dgrid = reinterpret_cast<long long*>(grid);
    else ok = ok && dalloc(&tmp, &dgrid, N3) == cudaSuccess;
    ok = ok && dalloc(&tmp, &dS, 1) == cudaSuccess && dalloc(&tmp, &dtot, 1) == cudaSuccess &&
         dalloc(&tmp, &dstep, 1) == cudaSuccess && dalloc(&tmp, &derr, 1) == cudaSuccess &&
         dalloc(&tmp, &dmax, 1) == cudaSuccess;
    if (!ok) {
        cleanup();
        return LC_ERR_OOM;
    }
    if (n_src > 0 && !pos_dev) e = cudaMemcpyAsync(dpos, pos, sizeof(double) * 3 * n_src, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && n_src > 0 && !lum_dev)
        e = cudaMemcpyAsync(dlum, lum, sizeof(double) * n_src, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dgrid, 0, sizeof(long long) * N3, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, sizeof(int), st);
    SlotMeta m{0, 0, dstep, dS, dtot};
    if (e == cudaSuccess) {
        launch_src_prep(dpos, dlum, n_src, dmax, derr, m, st);
        if (n_src > 0) launch_deposit(dpos, dlum, n_src, n, box / n, deposit, dmax, dgrid, m, derr, st);
        count_launch(n_src > 0 ? 2 : 1);
        e = cudaGetLastError();
    }
    long long tot = 0;
    double S = 1.0;
    int err = 0;
    if (e == cudaSuccess && !grid_dev)
        e = cudaMemcpyAsync(grid, dgrid, sizeof(long long) * N3, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&tot, dtot, sizeof(long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&S, dS, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, derr, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) return LC_ERR_CUDA;
    if (scale) *scale = S;
    if (total) *total = tot;
    return err ? LC_ERR_DEVICE_CHECK : LC_OK;
}

static lc_status fft_common(int n, cudaStream_t st, float2** work, float2** tw) {
    const FftOps* ops = ops_for(n);
    if (!ops) return LC_ERR_UNSUPPORTED_SIZE;
    if (ensure_init(ops) != cudaSuccess) return LC_ERR_CUDA;
    lc_plan tmp;
    const size_t spec = (size_t)n * n * nrp_of(n);
    if (dalloc(&tmp, work, spec) != cudaSuccess) return LC_ERR_OOM;
    if (dalloc(&tmp, tw, n) != cudaSuccess) {
        cudaFree(*work);
        return LC_ERR_OOM;
    }
    std::vector<float2> t = twiddles(n);
    if (cudaMemcpyAsync(*tw, t.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaFree(*work);
        cudaFree(*tw);
        return LC_ERR_CUDA;
    }
    return LC_OK;
}

lc_status lc_fft_r2c(int n, const float* in, float* out_complex, void* stream) {
    if (!in || !out_complex) return LC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    float2 *work = nullptr, *tw = nullptr;
    lc_status r = fft_common(n, st, &work, &tw);
    if (r != LC_OK) return r;
    const FftOps* ops = ops_for(n);
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
    ColsMaps maps;
    maps.make(work, n);
    const bool pl = ops->plane_r2c && ops->plane_on();
    if (pl) {
        ops->plane_r2c(ra, st);
    } else {
        ops->rows_r2c(ra, st);
        maps.set(c, nullptr);
        ops->cols(c, st);
    }
    c.axis = 1;
    maps.set(c, nullptr);
    ops->cols(c, st);
    count_launch(pl ? 2 : 3);
    const int h = n / 2 + 1;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(out_complex, sizeof(float2) * h, work, sizeof(float2) * nrp_of(n), sizeof(float2) * h,
                              (size_t)n * n, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(work);
    cudaFree(tw);
    return e == cudaSuccess ? LC_OK : LC_ERR_CUDA;
}

lc_status lc_fft_c2r(int n, const float* in_complex, float* out, float scale, void* stream) {
    if (!in_complex || !out) return LC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    float2 *work = nullptr, *tw = nullptr;
    lc_status r = fft_common(n, st, &work, &tw);
    if (r != LC_OK) return r;
    const FftOps* ops = ops_for(n);
    const int h = n / 2 + 1;
    cudaError_t e = cudaMemcpy2DAsync(work, sizeof(float2) * nrp_of(n), in_complex, sizeof(float2) * h,
                                      sizeof(float2) * h, (size_t)n * n, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) {
        ColArgs c{};
        c.axis = 1;
        c.dir = 1;
        c.in_mode = COL_IN_PLAIN;
        c.out_mode = COL_OUT_PLAIN;
        c.src = work;
        c.dst = work;
        c.tw = tw;
        ColsMaps maps;
        maps.make(work, n);
        maps.set(c, nullptr);
        ops->cols(c, st);
        c.axis = 0;
        maps.set(c, nullptr);
        RowC2RArgs ra{};
        ra.nrows = (long long)n * n;
        ra.src = work;
        ra.out = out;
        ra.scale = scale;
        ra.tw = tw;
        const bool pl = ops->plane_c2r && ops->plane_on();
        if (pl) {
            ops->plane_c2r(ra, st);
        } else {
            ops->cols(c, st);
            ops->rows_c2r(ra, st);
        }
        count_launch(pl ? 2 : 3);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(work);
    cudaFree(tw);
    return e == cudaSuccess ? LC_OK : LC_ERR_CUDA;
}

lc_status lc_batch_step(lc_plan* const* plans, int n, const int* steps, const int64_t* n_src,
                        const double* const* pos, const double* const* lum, float* const* outs) {
    if (!plans || n < 1 || !steps || !n_src || !outs) return LC_ERR_INVALID_ARG;
    // phase 1: every instance's deposit + forward transform; phase 2: every
    // instance's MAC + inverse transform.  Each plan runs on its own stream so
    // that the uneven instances overlap on the device.
    for (int i = 0; i < n; ++i) {
        if (n_src[i] < 0) continue;
        lc_status r = lc_push_sources(plans[i], steps[i], n_src[i], pos ? pos[i] : nullptr, lum ? lum[i] : nullptr);
        if (r != LC_OK) return r;
    }
    for (int i = 0; i < n; ++i) {
        lc_status r = lc_retarded_field(plans[i], steps[i], outs[i]);
        if (r != LC_OK) return r;
    }
    return LC_OK;
}

} // extern "C"
