// hd_ragged.cuh -- a ragged batch of 1D convolutions (different L, M, A, kind
// and parameters per instance) in one persistent kernel launch.
//
// The host turns the batch into a queue of tiles; persistent CTAs (one per SM)
// take tiles in queue order with an atomic counter:
//   FUSED  : up to G instances of one kernel configuration (S, kind, folded
//            blocks, mult, residue count), one thread group each (the fused
//            residue-at-a-time body of hd_conv1d.cuh);
//   COLFWD, ROW, COLBWD : the three phases of the split path (hd_split.cuh) for
//            one large instance, a block of columns or one row per tile.
// A split instance's ROW tiles wait for all its COLFWD tiles, its COLBWD tiles
// for all its ROW tiles, through per-instance counters (release by the
// producer, acquire by the consumer).  Split instances are packed into groups
// whose work buffers (A n S values each) share a small ring of buffers sized
// to stay in L2; the COLFWD tiles of group g wait until every COLBWD tile of
// group g - ring has finished with the buffer (a per-group counter).  Every
// consumer is queued after all of its producers, and a dequeued producer never
// waits on a later tile, so the waits always end; they are still bounded in
// time: a wait that exceeds the plan's limit records HD_ERR_TIMEOUT in an
// error word and skips its tile.
#pragma once

#include "hd_split.cuh"

namespace hd {

enum { RT_FUSED = 0, RT_COLFWD = 1, RT_ROW = 2, RT_COLBWD = 3 };

// one convolution of the ragged batch
struct RInst {
    const void* f[3];
    void* h;
    const void* twS;     // fused: FFT pass twiddles of (S, E); split: zeta_S^{j2 k1}
    const void* twN;     // residue twists
    const void* twS2;    // split: FFT pass twiddles of the row FFT (S2, 16)
    void* work;          // split: A n S values
    double invN;
    int L, Ls, H, n, N, S, S1, S2, A, ls_pad;
    int ncf, nrow, ncb;  // split: number of COLFWD / ROW / COLBWD tiles
    int grp;             // split: work-buffer group
    int gprev, gneed;    // split: group whose COLBWD tiles free the buffer, and their number (0: none)
    int stall;           // test hook: an extra, never-satisfied dependency
};

struct RTile {
    int type;
    int cfg;     // FUSED: configuration id; split: unused
    int first;   // FUSED: first position in the order array; split: instance
    int count;   // FUSED: instances in the tile; split: tile index within its phase
    int aux;     // FUSED: staged row length (max ls_pad of the tile)
    int pad0, pad1, pad2;
};

struct RaggedArgs {
    const RInst* inst;
    const RTile* tiles;
    const int* order;      // FUSED tiles: instance indices grouped by configuration
    int ntiles;
    int* head;             // queue position
    int* cnt1;             // per instance: finished COLFWD tiles
    int* cnt2;             // per instance: finished ROW tiles
    int* gdone;            // per split group: finished COLBWD tiles
    int* err;              // HD_ERR_TIMEOUT on a wait that ran out
    long long wait_ns;     // wait limit
};

__device__ __forceinline__ long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (long long)t;
}

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0 waits until *c >= target (or the limit passes); the CTA then agrees
// on the outcome.  Returns false (and records the timeout) if it ran out.
__device__ __forceinline__ bool cta_wait(const int* c, int target, const RaggedArgs& ra, int* flag) {
    if (threadIdx.x == 0) {
        int ok = 1;
        const long long t0 = global_ns();
        while (ld_acquire(c) < target) {
            if (global_ns() - t0 > ra.wait_ns) {
                atomicExch(ra.err, 5);
                ok = 0;
                break;
            }
            __nanosleep(200);
        }
        __threadfence();
        *flag = ok;
    }
    __syncthreads();
    const bool ok = *flag != 0;
    __syncthreads();
    return ok;
}

__device__ __forceinline__ void cta_signal(int* c) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(c, 1);
    }
}

__device__ __forceinline__ SplitArgs split_args_of(const RInst& r) {
    SplitArgs a;
    a.f[0] = r.f[0];
    a.f[1] = r.f[1];
    a.f[2] = r.f[2];
    for (int i = 3; i < kMaxIn; ++i) a.f[i] = nullptr;
    a.h[0] = r.h;   // one output (B = 1)
    for (int b = 1; b < kMaxOut; ++b) a.h[b] = nullptr;
    a.stride = 0;
    a.count = 1;
    a.L = r.L;
    a.Ls = r.Ls;
    a.H = r.H;
    a.n = r.n;
    a.S = r.S;
    a.S1 = r.S1;
    a.S2 = r.S2;
    a.A = r.A;
    a.B = 1;
    a.P = r.A;
    a.twS = r.twS;
    a.twR = r.twN;
    a.twS2 = r.twS2;
    a.work = r.work;
    a.invN = r.invN;
    a.r0 = 0;
    a.nr = r.n;
    a.accumulate = 0;
    return a;
}

__device__ __forceinline__ ConvArgs conv_args_of(const RInst& r) {
    ConvArgs a;
    a.f[0] = r.f[0];
    a.f[1] = r.f[1];
    a.f[2] = r.f[2];
    for (int i = 3; i < kMaxIn; ++i) a.f[i] = nullptr;
    a.h[0] = r.h;   // one output (B = 1)
    for (int b = 1; b < kMaxOut; ++b) a.h[b] = nullptr;
    a.stride = 0;
    a.count = 1;
    a.L = r.L;
    a.Ls = r.Ls;
    a.H = r.H;
    a.n = r.n;
    a.N = r.N;
    a.ls_pad = r.ls_pad;
    a.twS = r.twS;
    a.twN = r.twN;
    a.invN = r.invN;
    a.err = nullptr;
    a.r_begin = 0;
    a.r_end = r.n;
    return a;
}

}  // namespace hd
