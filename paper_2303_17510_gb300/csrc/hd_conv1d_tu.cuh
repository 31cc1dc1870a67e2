// hd_conv1d_tu.cuh -- instantiation table of the fused 1D kernels for one
// (dtype, kind, mult set).  Included by the hd_conv1d_<dtype>_<kind>[_b2].cu
// files with HD_REAL, HD_KIND, HD_DT, HD_KN, HD_VARIANTS and HD_UNIT_MULTS
// defined (HD_UNIT_MULTS(Y, ...) calls Y(mult, ...) for each mult of the unit).
#include <algorithm>
#include <cstdint>
#include <cstdlib>

#include "hd_dispatch.h"

namespace hd {

namespace {

template <class R, int S, int E, int MULT>
size_t group_smem(int ls_pad) {
    using MS = MultShape<MULT>;
    return (size_t(MS::A) * size_t(ls_pad) + size_t(MS::NX) * FftShape<S, E>::SMEM + size_t(MS::acc(S))) *
           sizeof(cplx<R>);
}

template <class R, int S, int E, int MULT>
int groups_for(int ls_pad) {
    const int T = S / E;
    int G = 256 / T;
    if (G < 1) G = 1;
    const size_t per = group_smem<R, S, E, MULT>(ls_pad);
    while (G > 1 && per * G > kMaxSmemPerBlock) --G;
    return per > kMaxSmemPerBlock ? 0 : G;
}

// error word of the persistent kernels of this unit (a bounded wait ran out)
__device__ int g_pipe_err;

int* pipe_err_ptr() {
    static int* ptrs[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!ptrs[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_pipe_err) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        ptrs[dev] = static_cast<int*>(p);
    }
    return ptrs[dev];
}

// Persistent CTAs with bulk-copy staging (conv1d_kernel_pipe), when every row
// is a whole number of 16-byte units on a 16-byte boundary: one staging buffer,
// released early (NBUF = 1; a second buffer for the one-CTA-per-SM variants
// measured 1.5 % slower on the 4096 x 4096 batch: the 64 KB it takes come out
// of the L1 that holds the twiddle tables).  HD_PIPE=0 turns the persistent
// kernels off.
template <class R, int S, int E, int KIND, int MULT, int NB, bool COMP, int MINB>
cudaError_t launch_pipe(const ConvArgs& a0, cudaStream_t st, bool* used) {
    constexpr int T = S / E;
    constexpr int A = MultShape<MULT>::A;
    constexpr int NX = MultShape<MULT>::NX;
    constexpr int NBUF = 1;
    *used = false;
    static const bool enabled = [] {
        const char* e = std::getenv("HD_PIPE");
        return !(e && e[0] == '0');
    }();
    if (!enabled) return cudaSuccess;
    const size_t esz = sizeof(cplx<R>);
    for (int aa = 0; aa < A; ++aa)
        if (reinterpret_cast<uintptr_t>(a0.f[aa]) % 16 != 0) return cudaSuccess;
    if ((a0.stride * esz) % 16 != 0 || (a0.Ls * esz) % 16 != 0 || (a0.ls_pad * esz) % 16 != 0) return cudaSuccess;
    int G = 256 / T;
    if (G < 1) G = 1;
    const size_t fft = (size_t(NX) * FftShape<S, E>::SMEM + size_t(MultShape<MULT>::acc(S))) * esz;
    const size_t stg = size_t(A) * a0.ls_pad * esz;
    while (G > 1 && G * (NBUF * stg + fft) > kMaxSmemPerBlock - 64) --G;
    const size_t smem = size_t(G) * (NBUF * stg + fft);
    if (smem > kMaxSmemPerBlock - 64) return cudaSuccess;
    auto k = conv1d_kernel_pipe<R, S, E, KIND, MULT, NB, COMP, MINB, NBUF>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cudaSuccess;
    }
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, G * T, smem) != cudaSuccess || per < MINB) {
        cudaGetLastError();
        return cudaSuccess;
    }
    ConvArgs a = a0;
    a.err = pipe_err_ptr();
    const int64_t steps = (a.count + G - 1) / G;
    if (steps <= 0) {
        *used = true;
        return cudaSuccess;
    }
    const int64_t grid = std::min<int64_t>(steps, (int64_t)sms * per);
    k<<<dim3((unsigned)grid), dim3(G * T), smem, st>>>(a);
    *used = true;
    return cudaGetLastError();
}

template <class R, int S, int E, int KIND, int MULT, int NB, bool COMP, int MINB>
cudaError_t launch_one(const ConvArgs& a, cudaStream_t st) {
    constexpr int T = S / E;
    // one convolution per CTA step (T >= 256) and plain sums: with smaller transforms the per-step
    // compute is too short to hide a copy (measured slower), and compensated sums (many residues)
    // are rare; both keep the plain kernel, which also bounds the instantiations
    if constexpr (!COMP && T >= 256) {
        bool used = false;
        cudaError_t e = launch_pipe<R, S, E, KIND, MULT, NB, COMP, MINB>(a, st, &used);
        if (used || e != cudaSuccess) return e;
    }
    const int G = groups_for<R, S, E, MULT>(a.ls_pad);
    if (G < 1) return cudaErrorInvalidValue;
    const size_t smem = size_t(G) * group_smem<R, S, E, MULT>(a.ls_pad);
    auto k = conv1d_kernel<R, S, E, KIND, MULT, NB, COMP, MINB>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int64_t blocks = (a.count + G - 1) / G;
    if (blocks <= 0) return cudaSuccess;
    k<<<dim3((unsigned)blocks), dim3(G * T), smem, st>>>(a);
    return cudaGetLastError();
}

template <class R, int S, int E, int KIND>
cudaError_t launch_fwd(const ConvArgs& a, int r, int m, void* out, cudaStream_t st) {
    const size_t smem = FftShape<S, E>::SMEM * sizeof(cplx<R>);
    auto k = forward_residue_kernel<R, S, E, KIND>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<1, S / E, smem, st>>>(a, r, m, out);
    return cudaGetLastError();
}

// Cluster variant: D residue groups x A inputs CTAs per convolution (complex
// and centered kinds, one output).  Shared memory: the staged row, one
// exchange buffer, two published spectra, the FFT twiddles and one twist row.
template <class R, int S, int E>
size_t cluster_smem(int ls_pad) {
    using Sh = FftShape<S, E>;
    return (size_t(ls_pad) + Sh::SMEM + 3 * size_t(S) + (Sh::TW_TOTAL > 0 ? Sh::TW_TOTAL : 1)) * sizeof(cplx<R>);
}

template <int MULT>
constexpr bool cluster_ok() {
    return HD_KIND != KIND_HERMITIAN && MultShape<MULT>::B == 1;
}

template <int S, int E, int MULT, int NB>
bool cluster_fits(int ls_pad, int D) {
    if constexpr (!cluster_ok<MULT>() || (HD_KIND == KIND_CENTERED && NB != 2)) {
        return false;
    } else {
        const int CL = D * MultShape<MULT>::A;
        return D >= 2 && CL <= 8 && cluster_smem<HD_REAL, S, E>(ls_pad) <= kMaxSmemPerBlock;
    }
}

template <int S, int E, int MULT, int NB>
cudaError_t launch_cluster(const ConvArgs& a, int D, cudaStream_t st) {
    if constexpr (!cluster_ok<MULT>() || (HD_KIND == KIND_CENTERED && NB != 2)) {
        return cudaErrorInvalidValue;
    } else {
        if (!cluster_fits<S, E, MULT, NB>(a.ls_pad, D)) return cudaErrorInvalidValue;
        if (a.count <= 0) return cudaSuccess;
        const int CL = D * MultShape<MULT>::A;
        const size_t smem = cluster_smem<HD_REAL, S, E>(a.ls_pad);
        auto k = conv1d_cluster_kernel<HD_REAL, S, E, HD_KIND, MULT, NB>;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(a.count * CL));
        cfg.blockDim = dim3(S / E);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)CL;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, k, a, D);
    }
}

// Hermitian data folds into one output block, centered data into two;
// compensated accumulation is an FP32 option.
template <int MULT, int NB, bool COMP>
constexpr bool combo_ok() {
    return !((HD_KIND == KIND_HERMITIAN && NB != 1) || (HD_KIND == KIND_CENTERED && NB != 2) ||
             (sizeof(HD_REAL) == 8 && COMP));
}

template <int S, int E, int MINB, int MULT, int NB, bool COMP>
cudaError_t pick(const ConvArgs& a, cudaStream_t st) {
    if constexpr (combo_ok<MULT, NB, COMP>()) return launch_one<HD_REAL, S, E, HD_KIND, MULT, NB, COMP, MINB>(a, st);
    else return cudaErrorInvalidValue;
}

template <int S, int E, int MINB, int MULT, int NB, bool COMP>
bool fits(int ls_pad) {
    if constexpr (combo_ok<MULT, NB, COMP>()) return groups_for<HD_REAL, S, E, MULT>(ls_pad) >= 1;
    else return false;
}

}  // namespace

// Kernel variants compiled for this dtype, as (S, E, MINB): HD_VARIANTS is
// defined by the including unit; every variant is compiled for each mult of
// the unit, both folded-block counts and both accumulations (combo_ok prunes).
#define HD_MULT_COMBOS(MU, SS, EE, MB, FN, ...)                                                          \
    if (c.mult == MU && c.nb == 1 && !c.comp) return FN<SS, EE, MB, MU, 1, false>(__VA_ARGS__);          \
    if (c.mult == MU && c.nb == 1 && c.comp) return FN<SS, EE, MB, MU, 1, true>(__VA_ARGS__);            \
    if (c.mult == MU && c.nb == 2 && !c.comp) return FN<SS, EE, MB, MU, 2, false>(__VA_ARGS__);          \
    if (c.mult == MU && c.nb == 2 && c.comp) return FN<SS, EE, MB, MU, 2, true>(__VA_ARGS__);
#define HD_COMBOS(SS, EE, MB, FN, ...)                                                                   \
    if (c.S == SS && c.E == EE && c.minb == MB) {                                                        \
        HD_UNIT_MULTS(HD_MULT_COMBOS, SS, EE, MB, FN, __VA_ARGS__)                                       \
    }

#define HD_LAUNCH_CASE(SS, EE, MB) HD_COMBOS(SS, EE, MB, pick, a, st)
#define HD_AVAIL_CASE(SS, EE, MB) HD_COMBOS(SS, EE, MB, fits, ls_pad)
#define HD_FWD_CASE(SS, EE, MB) \
    if (c.S == SS && c.E == EE) return launch_fwd<HD_REAL, SS, EE, HD_KIND>(a, r, m, out, st);
#define HD_LIST_CASE(SS, EE, MB) \
    if (n < cap) { out[n].S = SS; out[n].E = EE; out[n].minb = MB; } ++n;

#define HD_CAT2(a, b, c, d) a##b##c##d
#define HD_FN(base, DT, KN) HD_CAT2(base, DT, _, KN)

bool HD_FN(conv1d_available_, HD_DT, HD_KN)(const Conv1dCfg& c, int ls_pad) {
    HD_VARIANTS(HD_AVAIL_CASE)
    return false;
}

cudaError_t HD_FN(conv1d_launch_, HD_DT, HD_KN)(const Conv1dCfg& c, const ConvArgs& a, cudaStream_t st) {
    HD_VARIANTS(HD_LAUNCH_CASE)
    return cudaErrorInvalidValue;
}

cudaError_t HD_FN(forward_residue_launch_, HD_DT, HD_KN)(const Conv1dCfg& c, const ConvArgs& a, int r, int m,
                                                         void* out, cudaStream_t st) {
    HD_VARIANTS(HD_FWD_CASE)
    return cudaErrorInvalidValue;
}

#define HD_CLUSTER_MULT(MU, SS, EE, FN, ...)                                                          \
    if (c.mult == MU && c.nb == 1) return FN<SS, EE, MU, 1>(__VA_ARGS__);                              \
    if (c.mult == MU && c.nb == 2) return FN<SS, EE, MU, 2>(__VA_ARGS__);
#define HD_CLUSTER_FITS_CASE(SS, EE) \
    if (c.S == SS && c.E == EE) { HD_UNIT_MULTS(HD_CLUSTER_MULT, SS, EE, cluster_fits, ls_pad, D) }
#define HD_CLUSTER_LAUNCH_CASE(SS, EE) \
    if (c.S == SS && c.E == EE) { HD_UNIT_MULTS(HD_CLUSTER_MULT, SS, EE, launch_cluster, a, D, st) }

bool HD_FN(conv1d_cluster_available_, HD_DT, HD_KN)(const Conv1dCfg& c, int ls_pad, int D) {
    HD_CLUSTER_VARIANTS(HD_CLUSTER_FITS_CASE)
    return false;
}

cudaError_t HD_FN(conv1d_cluster_launch_, HD_DT, HD_KN)(const Conv1dCfg& c, const ConvArgs& a, int D,
                                                        cudaStream_t st) {
    HD_CLUSTER_VARIANTS(HD_CLUSTER_LAUNCH_CASE)
    return cudaErrorInvalidValue;
}

int HD_FN(conv1d_variants_, HD_DT, HD_KN)(Conv1dCfg* out, int cap) {
    int n = 0;
    HD_VARIANTS(HD_LIST_CASE)
    return n;
}

// Reads and clears this unit's error word on the current device (after the
// caller synchronized it): 1 if a bounded wait ran out, 0 if not, -1 on error.
int HD_FN(conv1d_take_error_, HD_DT, HD_KN)() {
    int v = 0;
    const int zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_pipe_err, sizeof(int)) != cudaSuccess ||
        cudaMemcpyToSymbol(g_pipe_err, &zero, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return v != 0 ? 1 : 0;
}

}  // namespace hd
