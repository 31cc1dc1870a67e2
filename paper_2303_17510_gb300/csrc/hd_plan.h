// hd_plan.h -- internal plan representation shared by the host sources.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <utility>
#include <vector>

#include "../../include/hd.h"
#include "hd_dispatch.h"

namespace hd {

enum { PATH_FUSED = 0, PATH_SPLIT = 1, PATH_COLUMN = 2 };

struct RaggedData;

// Makes `dev` the current device for the guard's lifetime (restores the
// caller's device afterwards).
struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
            changed = cudaSetDevice(dev) == cudaSuccess;
        }
    }
    ~DeviceGuard() {
        if (changed) cudaSetDevice(prev);
    }
    DeviceGuard(const DeviceGuard&) = delete;
    DeviceGuard& operator=(const DeviceGuard&) = delete;
};

// One axis of a plan: the paper's parameters (m, p, q, n, D) and the
// kernel geometry they map to (transform size S = m, p m or p m / 2;
// n residues of S values; nb folded blocks).
struct AxisPlan {
    int kind;
    int64_t L, M;      // logical length and dealiased length
    int64_t Ls;        // stored length (Hermitian: ceil(L/2))
    int64_t m, p, q, n, S;
    int D;
    int nb;
    int E;
    bool comp;         // compensated residue accumulation (FP32)
    int minb;          // kernel variant: CTAs per SM of the register allocation
    int path;
    void* twS;         // FUSED: FFT pass twiddles of (S, E); SPLIT: zeta_S^{j2 k1} (device)
    void* twN;         // residue twists, see upload_twists (device)
    void* twS2;        // SPLIT: FFT pass twiddles of the row FFT (device)
    int64_t S1, S2;    // SPLIT: S = S1 * S2
    int64_t chunk;     // SPLIT: instances per scratch chunk
};

// Residues per block of the split path: D when 1 < D < n (blocks accumulate
// into the output), else all n residues in one block.
inline int64_t split_block(const AxisPlan& ax) { return (ax.D > 1 && ax.D < ax.n) ? ax.D : ax.n; }

int64_t ceil_div(int64_t a, int64_t b);
int64_t next_pow2_t(int64_t x);   // smallest power of two >= x
bool is_pow2(int64_t x);
void zeta_fp64(int64_t k, int64_t N, double* c, double* s);
hd_status upload_zetas(const std::vector<std::pair<int64_t, int64_t>>& ek, int dtype, void** dev);
hd_status upload_fft_twiddles(int64_t S, int E, int dtype, void** dev);
hd_status upload_twists(int64_t S, int64_t n, int dtype, void** dev);
int max_fused_S(int dtype);
void axis_geometry(int kind, int64_t L, int64_t m, int64_t p, int64_t q, int64_t* S, int64_t* n, int* nb);
hd_status validate_axis(int kind, int mult, int64_t L, int64_t M, int64_t m, int64_t p, int64_t q, int64_t* S,
                        int64_t* n, int* nb);
bool fused_supported(int dtype, int kind, int mult, int64_t S, int nb, int64_t Ls, bool comp, int E, int minb);
// D > 1 residue groups of one convolution on a thread-block cluster (complex and
// centered kinds, one output): true when the cluster kernel runs the fused axis
bool cluster_supported(int dtype, int kind, int mult, int64_t S, int nb, int64_t Ls, int D, int E);
// default values per thread of the cluster variant: 4 for FP64 (see
// hd_conv1d_variants.h), 8 for FP32
inline int cluster_default_E(int dtype, int64_t S) { return dtype == HD_F64 && S <= 1024 ? 4 : 8; }
// candidates the learned selector and the ragged kernel consider: not the
// cluster variants (their features are those of the D = 1 candidate)
inline bool single_group(int kind, const hd_candidate& c) { return kind == HD_HERMITIAN || c.D <= 1; }
int default_minb(int dtype, int64_t S, int mult);
// split path (transforms larger than one CTA): S = S1 * S2, S2 the fused limit, S1 <= 16
bool split_supported(int dtype, int kind, int mult, int64_t S, int nb);
int64_t split_rows(int dtype);
hd_status upload_split_twiddles(int64_t S1, int64_t S2, int dtype, void** dev);
// staged row length in shared memory for Ls stored values (even: 16-byte rows)
inline int64_t staged_row(int64_t Ls) { return (Ls + 1) & ~int64_t(1); }
double cost_model(int kind, int A, int B, int64_t S, int64_t n);
// true when (A, B) are the input and output counts of the mult HD_MULT_*
bool mult_counts_ok(int mult, int A, int B);
// the kernels' mult (MULT_*) of a mult HD_MULT_*
int kernel_mult(int mult);

}  // namespace hd

struct hd_plan {
    int ndim;
    int kind;
    int dtype;
    int mult;
    int A, B;
    hd::AxisPlan ax[3];
    int64_t instance_elems;   // stored elements of one instance (all axes)
    size_t scratch_bytes;
    void* scratch;     // split-path work buffer (chunk * A * n * S values)
    void* work[2];     // N-D: work buffer of each outer axis level
    int64_t inst_cap;  // N-D: outer instances per pass through the levels
    int64_t level_chunk[2];   // N-D: instances of outer level k handled per pass (its work buffer's size)
    hd::RaggedData* ragged;   // ragged batch plans (hd_ragged.cu)
    int device;
    hd_status sticky;
};

namespace hd {

hd_status plan_create(hd_plan** out, const hd_desc* d);
hd_status plan_execute(hd_plan* plan, int64_t count, const void* const* f, void* const* h, int64_t stride,
                       cudaStream_t st);
// the partial sum over residues r_begin <= r < r_end of the outermost axis
// (0 <= r_begin < r_end <= n; 0, n is plan_execute)
hd_status plan_execute_range(hd_plan* plan, int64_t count, const void* const* f, void* const* h, int64_t stride,
                             int64_t r_begin, int64_t r_end, cudaStream_t st);
void plan_free(hd_plan* plan);
ConvArgs make_conv_args(const hd_plan& pl, const AxisPlan& ax, int64_t count, const void* const* f,
                        void* const* h, int64_t stride);
Conv1dCfg fused_cfg(const hd_plan& pl, const AxisPlan& ax);

hd_status fill_axis(int dtype, int kind, int mult, int64_t L, int64_t M, int64_t m, int64_t p, int64_t q, int D,
                    AxisPlan* ax);
// learned selector (hd_selector.cu)
void selector_features(const hd_desc* d, const hd_candidate* c, float* f);
bool selector_installed();
int selector_fallback();
hd_status selector_choose_batch(const std::vector<const hd_desc*>& descs,
                                const std::vector<std::vector<hd_candidate>>& cands, std::vector<int>* pick,
                                std::vector<int>* confident);
// timed search for one description, keeping candidates accepted by `ok`
hd_status timed_choice(const hd_desc* d, bool (*ok)(const hd_desc*, const hd_candidate&), hd_candidate* out);

// ragged batch plans (hd_ragged.cu)
hd_status ragged_create(hd_plan** out, int64_t n, const hd_desc* descs, const hd_candidate* forced);
void ragged_destroy(hd_plan* pl);
// multidimensional plans (hd_nd.cu)
hd_status plan_create_nd(hd_plan** out, const hd_desc* d);
hd_status plan_execute_nd(hd_plan* pl, int64_t count, const void* const* f, void* const* h, int64_t stride,
                          int64_t r_begin, int64_t r_end, cudaStream_t st);
// batched 1D convolution of rows with axis plan ax (fused or split path):
// the A inputs f, the B outputs h
hd_status rows_execute(const hd_plan& pl, const AxisPlan& ax, int64_t count, const void* const* f,
                       void* const* h, int64_t stride, void* scratch, cudaStream_t st);

// Plan for an explicit candidate (kernel variant included).
hd_status plan_create_from(hd_plan** out, const hd_desc* d, const hd_candidate* c);
bool comp_default(int64_t n);
// legal, supported candidates of a 1D description (see hd_enumerate_candidates)
int enumerate_candidates(const hd_desc* d, std::vector<hd_candidate>* out);
// tuned candidate recorded for the description, if any
bool cache_lookup(const hd_desc* d, hd_candidate* c);

// Split path over a caller-provided work buffer holding `chunk` instances.
hd_status split_execute(const hd_plan& pl, const AxisPlan& ax, int64_t count, const void* const* f, void* const* h,
                        int64_t stride, void* work, int64_t chunk, cudaStream_t st);
// the same for residues r_begin <= r < r_end only
hd_status split_execute_range(const hd_plan& pl, const AxisPlan& ax, int64_t count, const void* const* f,
                              void* const* h, int64_t stride, void* work, int64_t chunk, int64_t r_begin,
                              int64_t r_end, cudaStream_t st);

// Legal, supported (m, p, q) of one axis chosen by the cost model; fills ax.
hd_status choose_axis(int dtype, int kind, int mult, int A, int B, int64_t L, int64_t M, AxisPlan* ax);
// Axis parameters of a 1D description with m = 0: tuning cache, learned selector
// (timed search when unsure and allowed), cost model.
hd_status auto_axis(const hd_desc* d, AxisPlan* ax);

}  // namespace hd
