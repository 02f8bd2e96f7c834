// kbl_batch.cu -- the batched form: many independent 2D problems with uneven
// element counts and orders, advanced together.
//
// Every phase of a stage (time step, traces, bounds, residual, stage + limiter)
// is ONE persistent launch over all problems.  Each block pulls work items
// (problem, first element, element count) from a device counter; items are
// sorted by cost (order p, descending) so that the expensive ones start first
// and the tail is made of cheap ones.  The element code is the same device
// code the single-mesh kernels run (kbl_*_body.cuh), switched on the item's
// order.  A whole SSP-RK3 step is captured once as a CUDA graph (the counters
// are reset by a memset node).  The launch shape of the dominant bounds phase
// (thread tile, elements per item, resident blocks per SM) is chosen by
// kbl_batch_autotune, which times the candidates on a sample of the items.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "kbl_bounds_body.cuh"
#include "kbl_fr_body.cuh"
#include "kbl_limit_body.cuh"

namespace {

using namespace kbl_dev;

constexpr int PMAX_B = 4;        // orders 1..4
constexpr int NX_B = 32;         // velocity points per axis supported by the batch
constexpr int NTB = 256;         // threads per block of the FR / limiter phases
constexpr int FR_CHUNK = 256;    // elements per work item of the FR / limiter phases
constexpr int NCOUNTERS = 16;    // one work counter per persistent launch of a step
#define KBL_BATCH_HOST_GROUPS 8  // problem groups of kbl_batch_run_host (copies overlap steps)

struct ProbDesc {
    long long woff;     // state offset (doubles)
    long long wfoff;    // traces offset (doubles)
    long long bndoff;   // bounds offset (doubles)
    int E, p;
    int eoff;           // first element of the problem in the concatenated mesh
    int bcoff;          // first boundary state of the problem
    int n_bc;
};

struct WorkItem {
    int prob, e0, n;
};

struct BatchOps {
    FrOps o[PMAX_B + 1];     // index p
};

struct BatchDev {
    const ProbDesc* probs;
    const int* nbr;          // concatenated, local indices
    const double* h;
    const double* bc;
    int n_probs;
};

__device__ __forceinline__ MeshDev mesh_of_prob(const BatchDev& bd, const ProbDesc& pd)
{
    MeshDev m;
    m.E = pd.E;
    m.nbr = bd.nbr + (size_t)pd.eoff * 4;
    m.h = bd.h + (size_t)pd.eoff * 2;
    m.bc = bd.bc + (size_t)pd.bcoff * 4;
    m.n_bc = pd.n_bc;
    return m;
}

// Next work item of this block (block-uniform), or -1.
__device__ __forceinline__ int next_item(unsigned* counter, int n_items, int* s_item)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned it = atomicAdd(counter, 1u);
        *s_item = it < (unsigned)n_items ? (int)it : -1;
    }
    __syncthreads();
    return *s_item;
}

// ---------------------------------------------------------------------------
// persistent phase kernels
// ---------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ void traces_item(const ProbDesc& pd, const WorkItem& wi, const FrOps& ops,
                                            const double* __restrict__ w, double* __restrict__ wf)
{
    constexpr int NS = N * N, NFP = 4 * N;
    const double* wp = w + pd.woff;
    double* wfp = wf + pd.wfoff;
    for (int t = threadIdx.x; t < wi.n * NFP; t += blockDim.x) {
        const int e = wi.e0 + t / NFP, fp = t % NFP;
        const int f = fp / N, k = fp % N;
        const bool plus = f & 1, along_x = f < 2;
#pragma unroll
        for (int v = 0; v < 4; v++) {
            const double* we = wp + ((size_t)v * pd.E + e) * NS;
            double s = 0.0;
#pragma unroll
            for (int i = 0; i < N; i++) s += (plus ? ops.lp[i] : ops.lm[i]) * we[along_x ? k * N + i : i * N + k];
            wfp[((size_t)v * pd.E + e) * NFP + fp] = s;
        }
    }
}

__global__ void __launch_bounds__(NTB) k_batch_traces(BatchDev bd, const WorkItem* __restrict__ items, int n_items,
                                                      unsigned* counter, BatchOps ops, const double* w, double* wf)
{
    __shared__ int s_item;
    for (;;) {
        const int it = next_item(counter, n_items, &s_item);
        if (it < 0) break;
        const WorkItem wi = items[it];
        const ProbDesc pd = bd.probs[wi.prob];
        switch (pd.p) {
            case 1: traces_item<2>(pd, wi, ops.o[1], w, wf); break;
            case 2: traces_item<3>(pd, wi, ops.o[2], w, wf); break;
            case 3: traces_item<4>(pd, wi, ops.o[3], w, wf); break;
            case 4: traces_item<5>(pd, wi, ops.o[4], w, wf); break;
        }
    }
}

template <int TYSEL>
struct BoundsUnion {
    union {
        Bounds2dF32Smem<2, NX_B, TYSEL> s2;
        Bounds2dF32Smem<3, NX_B, TYSEL> s3;
        Bounds2dF32Smem<4, NX_B, TYSEL> s4;
        Bounds2dF32Smem<5, NX_B, TYSEL> s5;
    };
};

template <int N, int TYSEL>
__device__ __forceinline__ void bounds_item(void* smraw, const BatchDev& bd, const ProbDesc& pd, const WorkItem& wi,
                                            const Phys& ph, const double* w, const double* wf, double* bnd,
                                            DevFlags* flags)
{
    auto& sm = *reinterpret_cast<Bounds2dF32Smem<N, NX_B, TYSEL>*>(smraw);
    const MeshDev m = mesh_of_prob(bd, pd);
    for (int e = wi.e0; e < wi.e0 + wi.n; e++)
        bounds2d_f32_element<N, NX_B, TYSEL>(sm, w + pd.woff, wf + pd.wfoff, m, e, ph, bnd + pd.bndoff, flags);
}

// at least 7 resident blocks: the shared memory of a P4 work item allows 7, and without the
// hint the unrolled envelope loop takes enough registers to allow only 6
template <int TYSEL>
__global__ void __launch_bounds__(B2f32<NX_B, TYSEL>::NT, 7)
k_batch_bounds(BatchDev bd, const WorkItem* __restrict__ items, int n_items, unsigned* counter, Phys ph,
               const double* w, const double* wf, double* bnd, DevFlags* flags)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int s_item;
    for (;;) {
        const int it = next_item(counter, n_items, &s_item);
        if (it < 0) break;
        const WorkItem wi = items[it];
        const ProbDesc pd = bd.probs[wi.prob];
        switch (pd.p) {
            case 1: bounds_item<2, TYSEL>(smraw, bd, pd, wi, ph, w, wf, bnd, flags); break;
            case 2: bounds_item<3, TYSEL>(smraw, bd, pd, wi, ph, w, wf, bnd, flags); break;
            case 3: bounds_item<4, TYSEL>(smraw, bd, pd, wi, ph, w, wf, bnd, flags); break;
            case 4: bounds_item<5, TYSEL>(smraw, bd, pd, wi, ph, w, wf, bnd, flags); break;
        }
    }
}

template <int N, int NT = NTB>
struct FrEpb {
    static constexpr int EPB = NT / (N * N);
};

template <int NT = NTB>
struct RhsUnion {
    union {
        RhsSmem<2, 2, float, FrEpb<2, NT>::EPB> s2;
        RhsSmem<2, 3, float, FrEpb<3, NT>::EPB> s3;
        RhsSmem<2, 4, float, FrEpb<4, NT>::EPB> s4;
        RhsSmem<2, 5, float, FrEpb<5, NT>::EPB> s5;
    };
};

template <int N, int NT = NTB>
__device__ __forceinline__ void rhs_item(void* smraw, const BatchDev& bd, const ProbDesc& pd, const WorkItem& wi,
                                         const FrOps& ops, double gamma, int flux, const double* w, const double* wf,
                                         double* R)
{
    constexpr int EPB = FrEpb<N, NT>::EPB;
    auto& sm = *reinterpret_cast<RhsSmem<2, N, float, EPB>*>(smraw);
    const MeshDev m = mesh_of_prob(bd, pd);
    const int e_end = wi.e0 + wi.n;
    for (int eb = wi.e0; eb < e_end; eb += EPB)
        rhs_block<2, N, float, EPB>(sm, NT, w + pd.woff, wf + pd.wfoff, m, ops, gamma, R + pd.woff, eb,
                                    min(EPB, e_end - eb), flux);
}

// 4 resident blocks: without the hint the switch over orders inflates the register count
__global__ void __launch_bounds__(NTB, 4) k_batch_rhs(BatchDev bd, const WorkItem* __restrict__ items, int n_items,
                                                   unsigned* counter, BatchOps ops, double gamma, int flux,
                                                   const double* w, const double* wf, double* R)
{
    __shared__ __align__(16) RhsUnion<> sm;
    __shared__ int s_item;
    for (;;) {
        const int it = next_item(counter, n_items, &s_item);
        if (it < 0) break;
        const WorkItem wi = items[it];
        const ProbDesc pd = bd.probs[wi.prob];
        switch (pd.p) {
            case 1: rhs_item<2>(&sm, bd, pd, wi, ops.o[1], gamma, flux, w, wf, R); break;
            case 2: rhs_item<3>(&sm, bd, pd, wi, ops.o[2], gamma, flux, w, wf, R); break;
            case 3: rhs_item<4>(&sm, bd, pd, wi, ops.o[3], gamma, flux, w, wf, R); break;
            case 4: rhs_item<5>(&sm, bd, pd, wi, ops.o[4], gamma, flux, w, wf, R); break;
        }
    }
}

template <int NT = NTB>
struct LimUnion {
    union {
        LimSmem<2, 2, FrEpb<2, NT>::EPB> s2;
        LimSmem<2, 3, FrEpb<3, NT>::EPB> s3;
        LimSmem<2, 4, FrEpb<4, NT>::EPB> s4;
        LimSmem<2, 5, FrEpb<5, NT>::EPB> s5;
    };
};

template <int N, int NT = NTB>
__device__ __forceinline__ void stage_item(void* smraw, const ProbDesc& pd, const WorkItem& wi, const FrOps& ops,
                                           const Phys& ph, int stage, const double* wn, const double* ws,
                                           const double* R, const double* bnd, double dt, double* wout,
                                           DevFlags* flags)
{
    constexpr int EPB = FrEpb<N, NT>::EPB;
    auto& sm = *reinterpret_cast<LimSmem<2, N, EPB>*>(smraw);
    const int e_end = wi.e0 + wi.n;
    for (int eb = wi.e0; eb < e_end; eb += EPB)
        stage_limit_block<2, N, EPB>(sm, NT, 0, stage, wn + pd.woff, ws + pd.woff, R + pd.woff,
                                            bnd + pd.bndoff, dt, wout + pd.woff, nullptr, pd.E, ops, ph, flags, eb,
                                            min(EPB, e_end - eb));
}

// 4 resident blocks: without the hint the switch over orders inflates the register count
__global__ void __launch_bounds__(NTB, 4) k_batch_stage(BatchDev bd, const WorkItem* __restrict__ items, int n_items,
                                                     unsigned* counter, BatchOps ops, Phys ph, int stage,
                                                     const double* wn, const double* ws, const double* R,
                                                     const double* bnd, const double* dt, double* wout, DevFlags* flags)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int s_item;
    for (;;) {
        const int it = next_item(counter, n_items, &s_item);
        if (it < 0) break;
        const WorkItem wi = items[it];
        const ProbDesc pd = bd.probs[wi.prob];
        const double dtp = dt[wi.prob];
        switch (pd.p) {
            case 1: stage_item<2>(smraw, pd, wi, ops.o[1], ph, stage, wn, ws, R, bnd, dtp, wout, flags); break;
            case 2: stage_item<3>(smraw, pd, wi, ops.o[2], ph, stage, wn, ws, R, bnd, dtp, wout, flags); break;
            case 3: stage_item<4>(smraw, pd, wi, ops.o[3], ph, stage, wn, ws, R, bnd, dtp, wout, flags); break;
            case 4: stage_item<5>(smraw, pd, wi, ops.o[4], ph, stage, wn, ws, R, bnd, dtp, wout, flags); break;
        }
    }
}

// Per-problem time step: dtbits[prob] <- min of cfl h / (|U| + c) (FP32 arithmetic,
// as the single-mesh FP32-mixed path), then dt[prob] decoded.
template <int N>
__device__ __forceinline__ float dt_item(const BatchDev& bd, const ProbDesc& pd, const WorkItem& wi, float gamma,
                                         float cfl, const double* w)
{
    constexpr int NS = N * N;
    const double* wp = w + pd.woff;
    const double* h = bd.h + (size_t)pd.eoff * 2;
    float best = FLT_MAX;
    for (int t = threadIdx.x; t < wi.n * NS; t += blockDim.x) {
        const int e = wi.e0 + t / NS, nd = t % NS;
        float q[4];
#pragma unroll
        for (int v = 0; v < 4; v++) q[v] = from_f64<float>(wp[((size_t)v * pd.E + e) * NS + nd]);
        const float P = kbl_pressure<2, float>(q, gamma - 1.0f);
        const float a = sqrtf(gamma * P / q[0]);
#pragma unroll
        for (int k = 0; k < 2; k++)
            best = fminf(best, cfl * (from_f64<float>(h[e * 2 + k]) / (fabsf(q[1 + k] / q[0]) + a)));
    }
    return best;
}

__global__ void __launch_bounds__(NTB) k_batch_dt(BatchDev bd, const WorkItem* __restrict__ items, int n_items,
                                                  unsigned* counter, double gamma, double cfl,
                                                  const double* w, unsigned long long* dtbits)
{
    __shared__ int s_item;
    for (;;) {
        const int it = next_item(counter, n_items, &s_item);
        if (it < 0) break;
        const WorkItem wi = items[it];
        const ProbDesc pd = bd.probs[wi.prob];
        float b = FLT_MAX;
        switch (pd.p) {
            case 1: b = dt_item<2>(bd, pd, wi, (float)gamma, (float)cfl, w); break;
            case 2: b = dt_item<3>(bd, pd, wi, (float)gamma, (float)cfl, w); break;
            case 3: b = dt_item<4>(bd, pd, wi, (float)gamma, (float)cfl, w); break;
            case 4: b = dt_item<5>(bd, pd, wi, (float)gamma, (float)cfl, w); break;
        }
        unsigned long long bits = __double_as_longlong(to_f64<float>(b));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ob = __shfl_xor_sync(0xffffffffu, bits, o);
            bits = ob < bits ? ob : bits;
        }
        if ((threadIdx.x & 31) == 0) atomicMin(dtbits + wi.prob, bits);
    }
}

__global__ void k_batch_dt_finalize(const unsigned long long* dtbits, double* dt, double* t, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = __longlong_as_double((long long)dtbits[i]);
    if (!(v > 0.0) || !(v < DBL_MAX)) v = 0.0;
    dt[i] = v;
}

__global__ void k_batch_time_advance(const double* dt, double* t, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) t[i] += dt[i];
}

// ---------------------------------------------------------------------------
// The whole step as ONE persistent launch (dataflow).  The step's work is 13 phases -- the time
// step, then per stage s = 0, 1, 2: traces, bounds, residual, stage + limiter -- each cut into the
// same work items as the per-phase launches.  Blocks pull items from one counter in phase-major
// order; an item waits only until the earlier phases its problem depends on are complete (a
// per-problem count of finished items per phase), never on a grid-wide barrier, so the phases of
// different problems overlap.  Dependencies of a problem's phase: bounds and residual of stage s
// on its traces; the stage on its bounds and residual (stage 0 also on the time step); the traces
// of stage s + 1 on the stage s (which also releases the scratch the next stage rewrites).  An
// item depends only on items earlier in the queue, already taken by running blocks, so the
// launch cannot deadlock whatever the residency.  Waits poll with a bounded count; one that runs
// out raises the timeout flag and an abort word that ends every block at its next item.
// ---------------------------------------------------------------------------
constexpr int NTF = 128;   // threads per block of the fused step (the 4 x 2 or 2 x 4 bounds tile)
#ifndef KBL_FUSED_MINB
#define KBL_FUSED_MINB 7   // resident blocks per SM the fused kernel is compiled for (measured
                           // 5: 927, 6: 894, 7: 876 ms per step on the batched benchmark)
#endif
constexpr int NPH = 13;    // phases of a step
enum { PK_DT = 0, PK_TR = 1, PK_B = 2, PK_R = 3, PK_S = 4 };
__host__ __device__ __forceinline__ int phase_kind(int ph) { return ph == 0 ? PK_DT : 1 + (ph - 1) % 4; }
__host__ __device__ __forceinline__ int phase_stage(int ph) { return ph == 0 ? 0 : (ph - 1) / 4; }

struct FusedDev {
    const WorkItem* fr;    // FR / limiter / time-step items
    int n_fr;
    const WorkItem* bi;    // bounds items
    int n_b;
    const int* cnt_fr;     // [P] FR items of each problem
    const int* cnt_b;      // [P] bounds items of each problem
    unsigned* done;        // [NPH][P] finished items of each phase and problem (zeroed before the step)
    unsigned* queue;       // next item (zeroed before the step)
    int* abort;            // set when a wait ran out (zeroed before the step)
    int stall_test;        // nonzero: the first bounds item waits for a count no item reaches
    int wait_polls;        // bound of every wait, in polls of about 1 us
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Poll until *p >= target (bounded); false when the bound ran out or another block aborted.
__device__ __forceinline__ bool wait_count(const unsigned* p, unsigned target, int polls, const int* abort)
{
    for (int it = 0; it < polls; it++) {
        if (ld_acquire(p) >= target) return true;
        if (*(volatile const int*)abort) return false;
        __nanosleep(it < 16 ? 64 : 1024);
    }
    return ld_acquire(p) >= target;
}

template <int TYSEL>
struct FusedSmem {
    static constexpr size_t B = sizeof(BoundsUnion<TYSEL>), R_ = sizeof(RhsUnion<NTF>), L = sizeof(LimUnion<NTF>);
    static constexpr size_t BYTES = B > R_ ? (B > L ? B : L) : (R_ > L ? R_ : L);
};

template <int TYSEL>
__global__ void __launch_bounds__(NTF, KBL_FUSED_MINB)
k_batch_step_fused(BatchDev bd, FusedDev fd, BatchOps ops, Phys ph, double cfl, double* w, double* wa, double* wb,
                   double* wf, double* R, double* bnd, unsigned long long* dtbits, double* dtv, double* tv,
                   DevFlags* flags)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ int s_item, s_ok;
    const int P = bd.n_probs;
    const int total = 10 * fd.n_fr + 3 * fd.n_b;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned it = atomicAdd(fd.queue, 1u);
            s_item = (it < (unsigned)total && !*(volatile int*)fd.abort) ? (int)it : -1;
        }
        __syncthreads();
        int idx = s_item;
        if (idx < 0) break;
        int phs = 0;
        for (; phs < NPH - 1; phs++) {
            const int n = phase_kind(phs) == PK_B ? fd.n_b : fd.n_fr;
            if (idx < n) break;
            idx -= n;
        }
        const int kind = phase_kind(phs), st = phase_stage(phs);
        const WorkItem wi = kind == PK_B ? fd.bi[idx] : fd.fr[idx];
        const int prob = wi.prob;
        // dependencies (thread 0 waits; the block follows)
        if (threadIdx.x == 0) {
            bool ok = true;
            const unsigned nfr = (unsigned)fd.cnt_fr[prob], nb = (unsigned)fd.cnt_b[prob];
            if (kind == PK_TR && st > 0) ok = wait_count(fd.done + (size_t)(phs - 1) * P + prob, nfr, fd.wait_polls, fd.abort);
            if (kind == PK_B) {
                const unsigned extra = (fd.stall_test && phs == 2 && idx == 0) ? 1u : 0u;   // a count never reached
                ok = wait_count(fd.done + (size_t)(phs - 1) * P + prob, nfr + extra, fd.wait_polls, fd.abort);
            }
            if (kind == PK_R) ok = wait_count(fd.done + (size_t)(phs - 2) * P + prob, nfr, fd.wait_polls, fd.abort);
            if (kind == PK_S) {
                ok = wait_count(fd.done + (size_t)(phs - 2) * P + prob, nb, fd.wait_polls, fd.abort) &&
                     wait_count(fd.done + (size_t)(phs - 1) * P + prob, nfr, fd.wait_polls, fd.abort);
                if (ok && st == 0) ok = wait_count(fd.done + prob, nfr, fd.wait_polls, fd.abort);
            }
            if (!ok) {
                if (!*(volatile int*)fd.abort) atomicOr(&flags->timeout, 1);
                atomicExch(fd.abort, 1);
            }
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) break;
        __threadfence();
        const ProbDesc pd = bd.probs[prob];
        // stage inputs and outputs: w -> wa -> wb -> w (selects, not an indexed array)
        const double* ws = st == 0 ? w : (st == 1 ? wa : wb);
        double* wo = st == 0 ? wa : (st == 1 ? wb : w);
        if (kind == PK_DT) {
            float b = FLT_MAX;
            switch (pd.p) {
                case 1: b = dt_item<2>(bd, pd, wi, (float)ph.gamma, (float)cfl, w); break;
                case 2: b = dt_item<3>(bd, pd, wi, (float)ph.gamma, (float)cfl, w); break;
                case 3: b = dt_item<4>(bd, pd, wi, (float)ph.gamma, (float)cfl, w); break;
                case 4: b = dt_item<5>(bd, pd, wi, (float)ph.gamma, (float)cfl, w); break;
            }
            unsigned long long bits = __double_as_longlong(to_f64<float>(b));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long ob = __shfl_xor_sync(0xffffffffu, bits, o);
                bits = ob < bits ? ob : bits;
            }
            if ((threadIdx.x & 31) == 0) atomicMin(dtbits + prob, bits);
        } else if (kind == PK_TR) {
            switch (pd.p) {
                case 1: traces_item<2>(pd, wi, ops.o[1], ws, wf); break;
                case 2: traces_item<3>(pd, wi, ops.o[2], ws, wf); break;
                case 3: traces_item<4>(pd, wi, ops.o[3], ws, wf); break;
                case 4: traces_item<5>(pd, wi, ops.o[4], ws, wf); break;
            }
        } else if (kind == PK_B) {
            switch (pd.p) {
                case 1: bounds_item<2, TYSEL>(smraw, bd, pd, wi, ph, ws, wf, bnd, flags); break;
                case 2: bounds_item<3, TYSEL>(smraw, bd, pd, wi, ph, ws, wf, bnd, flags); break;
                case 3: bounds_item<4, TYSEL>(smraw, bd, pd, wi, ph, ws, wf, bnd, flags); break;
                case 4: bounds_item<5, TYSEL>(smraw, bd, pd, wi, ph, ws, wf, bnd, flags); break;
            }
        } else if (kind == PK_R) {
            switch (pd.p) {
                case 1: rhs_item<2, NTF>(smraw, bd, pd, wi, ops.o[1], ph.gamma, ph.flux, ws, wf, R); break;
                case 2: rhs_item<3, NTF>(smraw, bd, pd, wi, ops.o[2], ph.gamma, ph.flux, ws, wf, R); break;
                case 3: rhs_item<4, NTF>(smraw, bd, pd, wi, ops.o[3], ph.gamma, ph.flux, ws, wf, R); break;
                case 4: rhs_item<5, NTF>(smraw, bd, pd, wi, ops.o[4], ph.gamma, ph.flux, ws, wf, R); break;
            }
        } else {
            // the problem's time step (all its time-step items are complete): k_batch_dt_finalize's decoding
            double dtp = __longlong_as_double((long long)atomicAdd(dtbits + prob, 0ull));
            if (!(dtp > 0.0) || !(dtp < DBL_MAX)) dtp = 0.0;
            switch (pd.p) {
                case 1: stage_item<2, NTF>(smraw, pd, wi, ops.o[1], ph, st, w, ws, R, bnd, dtp, wo, flags); break;
                case 2: stage_item<3, NTF>(smraw, pd, wi, ops.o[2], ph, st, w, ws, R, bnd, dtp, wo, flags); break;
                case 3: stage_item<4, NTF>(smraw, pd, wi, ops.o[3], ph, st, w, ws, R, bnd, dtp, wo, flags); break;
                case 4: stage_item<5, NTF>(smraw, pd, wi, ops.o[4], ph, st, w, ws, R, bnd, dtp, wo, flags); break;
            }
            if (st == 2) {
                __syncthreads();
                if (threadIdx.x == 0) {
                    __threadfence();
                    // the problem's last stage-2 item: publish its time step and advance its clock
                    if (atomicAdd(fd.done + (size_t)phs * P + prob, 1u) + 1u == (unsigned)fd.cnt_fr[prob]) {
                        dtv[prob] = dtp;
                        tv[prob] += dtp;
                    }
                }
                continue;
            }
        }
        // publish: this item's writes before its count
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(fd.done + (size_t)phs * P + prob, 1u);
        }
    }
}

}  // namespace

// ===========================================================================
// host side
// ===========================================================================
struct kbl_batch {
    kbl_config cfg;
    Phys phys;
    BatchOps ops;
    cudaStream_t stream = nullptr;
    int P = 0;
    long long E_total = 0, W_total = 0, WF_total = 0, BND_total = 0;
    std::vector<ProbDesc> probs;
    std::vector<WorkItem> fr_items_h;
    ProbDesc* d_probs = nullptr;
    int* d_nbr = nullptr;
    double* d_h = nullptr;
    double* d_bc = nullptr;
    double *d_wf = nullptr, *d_R = nullptr, *d_bnd = nullptr, *d_wa = nullptr, *d_wb = nullptr;
    double *d_dt = nullptr, *d_t = nullptr;
    unsigned long long* d_dtbits = nullptr;
    DevFlags* d_flags = nullptr;
    unsigned* d_counters = nullptr;
    WorkItem* d_fr_items = nullptr;
    int n_fr_items = 0;
    WorkItem* d_b_items = nullptr;       // bounds items for the current chunk size
    int n_b_items = 0;
    // launch shape of the bounds phase
    int tile = 0, chunk = 16, blocks_per_sm = 0;
    int nsm = 0;
    // graph of kbl_batch_step
    cudaGraphExec_t graph = nullptr;
    double* graph_w = nullptr;
    double graph_cfl = 0.0;
    int graph_kernels = 0;
    int64_t launches = 0;
    std::string err;
    // kbl_batch_run_host: the library's device copy of the state and the problems cut into
    // groups of consecutive problems, each with its own work items, counters and step graph, so
    // that the copies of one group overlap the step of another
    struct Group {
        int p0 = 0, p1 = 0;
        WorkItem* fr = nullptr;
        int n_fr = 0;
        WorkItem* bi = nullptr;
        int n_bi = 0, chunk = 0;
        cudaGraphExec_t graph = nullptr;
        double cfl = 0.0;
        int kernels = 0;
        cudaEvent_t h2d = nullptr, done = nullptr;
    };
    std::vector<Group> groups;
    double* d_whost = nullptr;
    unsigned* d_gcounters = nullptr;
    cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
    // timing of the bounds launch of kbl_batch_bounds (kbl_batch_bounds_ms)
    cudaEvent_t tb0 = nullptr, tb1 = nullptr;
    bool tb_valid = false;
    // the fused single-launch step (kbl_batch_set_form) and its control words
    int fused = 0;
    int stall_test = 0;
    int wait_polls = 1 << 20;          // about a second per wait
    int* d_cnt = nullptr;              // [2][P]: FR items, bounds items of each problem
    unsigned* d_done = nullptr;        // [13][P] finished items per phase and problem
    unsigned* d_fctl = nullptr;        // [0] queue, [1] abort; per group g at 2 + 2 g
};

namespace {

kbl_status bfail(kbl_batch* b, kbl_status st, const std::string& msg)
{
    if (b) b->err = msg;
    return st;
}

// launch-shape tile index -> thread tile of the bounds body: 0 = 4x4 (64 threads), 1 = 4x2, 2 = 2x4
// (128 threads each)
size_t bounds_smem(int tile)
{
    return tile == 2 ? sizeof(BoundsUnion<3>) : tile == 1 ? sizeof(BoundsUnion<2>) : sizeof(BoundsUnion<0>);
}

std::vector<WorkItem> make_items(const std::vector<ProbDesc>& probs, int chunk, int p0 = 0, int p1 = -1)
{
    std::vector<WorkItem> items;
    if (p1 < 0) p1 = (int)probs.size();
    for (int pi = p0; pi < p1; pi++)
        for (int e0 = 0; e0 < probs[pi].E; e0 += chunk) items.push_back({pi, e0, std::min(chunk, probs[pi].E - e0)});
    // expensive first: higher order, then fuller items
    std::stable_sort(items.begin(), items.end(), [&](const WorkItem& a, const WorkItem& b) {
        const int pa = probs[a.prob].p, pb = probs[b.prob].p;
        if (pa != pb) return pa > pb;
        return a.n > b.n;
    });
    return items;
}

cudaError_t upload_items(kbl_batch* b, const std::vector<WorkItem>& items, WorkItem** d, int* n)
{
    if (*d) cudaFree(*d);
    *d = nullptr;
    *n = (int)items.size();
    cudaError_t e = cudaMalloc((void**)d, std::max<size_t>(1, items.size()) * sizeof(WorkItem));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*d, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice);
}

BatchDev dev_of(const kbl_batch* b)
{
    BatchDev bd;
    bd.probs = b->d_probs;
    bd.nbr = b->d_nbr;
    bd.h = b->d_h;
    bd.bc = b->d_bc;
    bd.n_probs = b->P;
    return bd;
}

int grid_of(const kbl_batch* b, int per_sm) { return std::max(1, b->nsm * std::max(1, per_sm)); }

// Bounds phase on (w, wf) -> bnd with the current launch shape; work counter `counter`.
int launch_bounds_phase(kbl_batch* b, const double* w, const double* wf, double* bnd, unsigned* counter,
                        cudaStream_t s, const WorkItem* items, int n_items)
{
    const BatchDev bd = dev_of(b);
    const size_t smem = bounds_smem(b->tile);
    const int grid = grid_of(b, b->blocks_per_sm);
    if (b->tile == 2)
        k_batch_bounds<3><<<grid, B2f32<NX_B, 3>::NT, smem, s>>>(bd, items, n_items, counter, b->phys, w, wf, bnd,
                                                                  b->d_flags);
    else if (b->tile)
        k_batch_bounds<2><<<grid, B2f32<NX_B, 2>::NT, smem, s>>>(bd, items, n_items, counter, b->phys, w, wf, bnd,
                                                                  b->d_flags);
    else
        k_batch_bounds<0><<<grid, B2f32<NX_B, 0>::NT, smem, s>>>(bd, items, n_items, counter, b->phys, w, wf, bnd,
                                                                  b->d_flags);
    return 1;
}

int fr_blocks_per_sm(const void* fn, size_t smem)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, NTB, smem) != cudaSuccess || n < 1) n = 1;
    return n;
}

// The work of one step: FR and bounds work items of problems [p0, p1) and the counter slots of
// its persistent launches.
struct ItemSet {
    const WorkItem* fr;
    int n_fr;
    const WorkItem* bi;
    int n_bi;
    unsigned* counters;
    int p0, p1;
};

ItemSet all_items(const kbl_batch* b)
{
    return {b->d_fr_items, b->n_fr_items, b->d_b_items, b->n_b_items, b->d_counters, 0, b->P};
}

// One SSP-RK3 step of the problems of `is` on stream s (also used for capture).
// One step of the item set as per-phase persistent launches.  With a side stream s2 and its
// events, each stage's residual runs on a branch of its own beside the stage's bounds (both read
// only the stage input and its traces); the stage kernel waits for both.
int issue_batch_step(kbl_batch* b, double* w, double cfl, cudaStream_t s, const ItemSet& is,
                     cudaStream_t s2 = nullptr, cudaEvent_t* ev = nullptr)
{
    const BatchDev bd = dev_of(b);
    const int np = is.p1 - is.p0;
    int n = 0;
    cudaMemsetAsync(is.counters, 0, NCOUNTERS * sizeof(unsigned), s);
    cudaMemsetAsync(b->d_dtbits + is.p0, 0x7f, (size_t)np * sizeof(unsigned long long), s);
    const int g_tr = grid_of(b, fr_blocks_per_sm((const void*)k_batch_traces, 0));
    const int g_rhs = grid_of(b, fr_blocks_per_sm((const void*)k_batch_rhs, 0));
    const int g_st = grid_of(b, fr_blocks_per_sm((const void*)k_batch_stage, sizeof(LimUnion<>)));
    const int g_dt = grid_of(b, fr_blocks_per_sm((const void*)k_batch_dt, 0));
    k_batch_dt<<<g_dt, NTB, 0, s>>>(bd, is.fr, is.n_fr, is.counters + 0, b->phys.gamma, cfl, w, b->d_dtbits);
    k_batch_dt_finalize<<<(np + 255) / 256, 256, 0, s>>>(b->d_dtbits + is.p0, b->d_dt + is.p0, b->d_t + is.p0, np);
    n += 2;
    const double* wn = w;
    const double* ws = w;
    double* outs[3] = {b->d_wa, b->d_wb, w};
    for (int st = 0; st < 3; st++) {
        k_batch_traces<<<g_tr, NTB, 0, s>>>(bd, is.fr, is.n_fr, is.counters + 1 + 4 * st, b->ops, ws, b->d_wf);
        cudaStream_t sr = s;
        if (s2) {
            cudaEventRecord(ev[2 * st], s);
            cudaStreamWaitEvent(s2, ev[2 * st], 0);
            sr = s2;
        }
        k_batch_rhs<<<g_rhs, NTB, 0, sr>>>(bd, is.fr, is.n_fr, is.counters + 3 + 4 * st, b->ops, b->phys.gamma,
                                           b->phys.flux, ws, b->d_wf, b->d_R);
        if (s2) cudaEventRecord(ev[2 * st + 1], s2);
        n += launch_bounds_phase(b, ws, b->d_wf, b->d_bnd, is.counters + 2 + 4 * st, s, is.bi, is.n_bi);
        if (s2) cudaStreamWaitEvent(s, ev[2 * st + 1], 0);
        k_batch_stage<<<g_st, NTB, sizeof(LimUnion<>), s>>>(bd, is.fr, is.n_fr, is.counters + 4 + 4 * st, b->ops,
                                                          b->phys, st, wn, ws, b->d_R, b->d_bnd, b->d_dt, outs[st],
                                                          b->d_flags);
        n += 3;
        ws = outs[st];
    }
    k_batch_time_advance<<<(np + 255) / 256, 256, 0, s>>>(b->d_dt + is.p0, b->d_t + is.p0, np);
    return n + 1;
}

int issue_batch_step_fused(kbl_batch* b, double* w, double cfl, cudaStream_t s, const ItemSet& is, unsigned* ctl);

// Capture one step of `is` on state w as a graph.
cudaError_t capture_step(kbl_batch* b, double* w, double cfl, const ItemSet& is, cudaGraphExec_t* out, int* kernels)
{
    *out = nullptr;
    cudaStream_t cap = nullptr, side = nullptr;
    cudaEvent_t ev[6] = {};
    int prio_lo = 0, prio_hi = 0;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (e == cudaSuccess && !b->fused) e = cudaStreamCreateWithPriority(&side, cudaStreamNonBlocking, prio_hi);
    for (int k = 0; k < 6 && e == cudaSuccess && side; k++) e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
    auto release = [&]() {
        for (int k = 0; k < 6; k++)
            if (ev[k]) cudaEventDestroy(ev[k]);
        if (side) cudaStreamDestroy(side);
        if (cap) cudaStreamDestroy(cap);
    };
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        release();
        return e;
    }
    *kernels = b->fused ? issue_batch_step_fused(b, w, cfl, cap, is, is.counters)
                        : issue_batch_step(b, w, cfl, cap, is, side, ev);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cap, &g);
    release();
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) *out = nullptr;
    return e;
}

void drop_groups(kbl_batch* b)
{
    for (auto& g : b->groups) {
        if (g.graph) cudaGraphExecDestroy(g.graph);
        if (g.fr) cudaFree(g.fr);
        if (g.bi) cudaFree(g.bi);
        if (g.h2d) cudaEventDestroy(g.h2d);
        if (g.done) cudaEventDestroy(g.done);
    }
    b->groups.clear();
}

// Items per problem (FR and bounds) for the fused step's dependency counts.
cudaError_t upload_counts(kbl_batch* b)
{
    std::vector<int> cnt(2 * (size_t)b->P, 0);
    for (int i = 0; i < b->P; i++) {
        cnt[i] = (b->probs[i].E + FR_CHUNK - 1) / FR_CHUNK;
        cnt[b->P + i] = (b->probs[i].E + b->chunk - 1) / b->chunk;
    }
    cudaError_t e = cudaSuccess;
    if (!b->d_cnt) e = cudaMalloc((void**)&b->d_cnt, cnt.size() * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_cnt, cnt.data(), cnt.size() * sizeof(int), cudaMemcpyHostToDevice);
    return e;
}

template <int TYSEL>
int fused_blocks_per_sm()
{
    int n = 0;
    const size_t smem = FusedSmem<TYSEL>::BYTES;
    cudaFuncSetAttribute(k_batch_step_fused<TYSEL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_step_fused<TYSEL>, NTF, smem);
    return std::max(1, n);
}

// One SSP-RK3 step of the problems of `is` as ONE kernel launch (plus the resets of its control
// words); ctl: [queue, abort] of this launch.
int issue_batch_step_fused(kbl_batch* b, double* w, double cfl, cudaStream_t s, const ItemSet& is, unsigned* ctl)
{
    const int np = is.p1 - is.p0;
    cudaMemsetAsync(ctl, 0, 2 * sizeof(unsigned), s);
    cudaMemsetAsync(b->d_done, 0, (size_t)NPH * b->P * sizeof(unsigned), s);
    cudaMemsetAsync(b->d_dtbits + is.p0, 0x7f, (size_t)np * sizeof(unsigned long long), s);
    FusedDev fd;
    fd.fr = is.fr;
    fd.n_fr = is.n_fr;
    fd.bi = is.bi;
    fd.n_b = is.n_bi;
    fd.cnt_fr = b->d_cnt;
    fd.cnt_b = b->d_cnt + b->P;
    fd.done = b->d_done;
    fd.queue = ctl;
    fd.abort = reinterpret_cast<int*>(ctl + 1);
    fd.stall_test = b->stall_test;
    fd.wait_polls = b->wait_polls;
    const BatchDev bd = dev_of(b);
    if (b->tile == 2) {
        const int grid = b->nsm * std::min(fused_blocks_per_sm<3>(), std::max(1, b->blocks_per_sm));
        k_batch_step_fused<3><<<grid, NTF, FusedSmem<3>::BYTES, s>>>(bd, fd, b->ops, b->phys, cfl, w, b->d_wa, b->d_wb,
                                                                   b->d_wf, b->d_R, b->d_bnd, b->d_dtbits, b->d_dt,
                                                                   b->d_t, b->d_flags);
    } else {
        const int grid = b->nsm * std::min(fused_blocks_per_sm<2>(), std::max(1, b->blocks_per_sm));
        k_batch_step_fused<2><<<grid, NTF, FusedSmem<2>::BYTES, s>>>(bd, fd, b->ops, b->phys, cfl, w, b->d_wa, b->d_wb,
                                                                   b->d_wf, b->d_R, b->d_bnd, b->d_dtbits, b->d_dt,
                                                                   b->d_t, b->d_flags);
    }
    return 1;
}

void drop_graph(kbl_batch* b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_w = nullptr;
}

cudaError_t set_bounds_shape(kbl_batch* b, int tile, int chunk, int per_sm)
{
    b->tile = tile;
    b->blocks_per_sm = per_sm;
    if (chunk != b->chunk || !b->d_b_items) {
        b->chunk = chunk;
        cudaError_t e = upload_items(b, make_items(b->probs, chunk), &b->d_b_items, &b->n_b_items);
        if (e == cudaSuccess) e = upload_counts(b);
        if (e != cudaSuccess) return e;
    }
    drop_graph(b);
    drop_groups(b);
    return cudaSuccess;
}

int max_bounds_blocks(int tile)
{
    int n = 0;
    const size_t smem = bounds_smem(tile);
    if (tile == 2) {
        cudaFuncSetAttribute(k_batch_bounds<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_bounds<3>, B2f32<NX_B, 3>::NT, smem);
    } else if (tile) {
        cudaFuncSetAttribute(k_batch_bounds<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_bounds<2>, B2f32<NX_B, 2>::NT, smem);
    } else {
        cudaFuncSetAttribute(k_batch_bounds<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_bounds<0>, B2f32<NX_B, 0>::NT, smem);
    }
    return std::max(1, n);
}

}  // namespace

extern "C" {

kbl_status kbl_batch_create(kbl_batch** out, const kbl_config* cfg, int P, const int32_t* p, const int32_t* n_elem,
                            const int32_t* nbr, const double* h, const int32_t* n_bc, const double* bc,
                            void* cuda_stream)
{
    if (!out) return KBL_EINVAL;
    *out = nullptr;
    if (!cfg || cfg->dim != 2 || cfg->precision != KBL_FP32_MIXED || cfg->nu[0] != NX_B || cfg->nu[1] != NX_B)
        return KBL_EINVAL;
    if (!(cfg->gamma > 1.0) || !(cfg->k > 0.0) || !(cfg->r_fac >= 0.0 && cfg->r_fac < 1.0) || !(cfg->eps >= 0.0))
        return KBL_EINVAL;
    if (cfg->flux < 0 || cfg->flux > 2 || cfg->quadrature != 0 || cfg->stencil != 0) return KBL_EINVAL;
    if (P < 1 || !p || !n_elem || !nbr || !h || !n_bc) return KBL_EINVAL;
    kbl_batch* b = new (std::nothrow) kbl_batch();
    if (!b) return KBL_ENOMEM;
    b->cfg = *cfg;
    b->stream = (cudaStream_t)cuda_stream;
    b->phys.gamma = cfg->gamma;
    b->phys.k = cfg->k;
    b->phys.r_fac = cfg->r_fac;
    b->phys.eps = cfg->eps;
    b->phys.rho_floor = cfg->rho_floor;
    b->phys.p_floor = cfg->p_floor;
    b->phys.eps_rule = cfg->eps_rule;
    b->phys.uncoupled = cfg->uncoupled ? 1 : 0;
    b->phys.flux = cfg->flux;
    b->phys.qw = nullptr;
    b->phys.qwf = nullptr;
    b->phys.nu[0] = b->phys.nu[1] = NX_B;
    kbl_phys_derive(b->phys);
    for (int q = 1; q <= PMAX_B; q++) kbl_build_fr_ops(q, b->ops.o[q]);
    b->P = P;
    long long eoff = 0, bcoff = 0, woff = 0, wfoff = 0, bndoff = 0;
    for (int i = 0; i < P; i++) {
        if (p[i] < 1 || p[i] > PMAX_B || n_elem[i] < 1 || n_bc[i] < 0) {
            delete b;
            return KBL_EINVAL;
        }
        const int n = p[i] + 1, E = n_elem[i];
        for (long long k = 0; k < (long long)E * 4; k++) {
            const int v = nbr[eoff * 4 + k];
            if (v >= E || (v < 0 && -(v + 1) >= n_bc[i])) {
                delete b;
                return KBL_EINVAL;
            }
        }
        for (long long k = 0; k < (long long)E * 2; k++)
            if (!(h[eoff * 2 + k] > 0.0)) {
                delete b;
                return KBL_EINVAL;
            }
        ProbDesc d;
        d.woff = woff;
        d.wfoff = wfoff;
        d.bndoff = bndoff;
        d.E = E;
        d.p = p[i];
        d.eoff = (int)eoff;
        d.bcoff = (int)bcoff;
        d.n_bc = n_bc[i];
        b->probs.push_back(d);
        woff += 4LL * E * n * n;
        wfoff += 4LL * E * 4 * n;
        bndoff += 8LL * E;
        eoff += E;
        bcoff += n_bc[i];
    }
    if (eoff > 0x7fffffffLL) {
        delete b;
        return KBL_EINVAL;
    }
    b->E_total = eoff;
    b->W_total = woff;
    b->WF_total = wfoff;
    b->BND_total = bndoff;
    cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, 0);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaSuccess;
    auto A = [&](void** ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, std::max<size_t>(bytes, 16));
    };
    A((void**)&b->d_probs, P * sizeof(ProbDesc));
    A((void**)&b->d_nbr, eoff * 4 * sizeof(int));
    A((void**)&b->d_h, eoff * 2 * sizeof(double));
    A((void**)&b->d_bc, std::max<long long>(bcoff, 1) * 4 * sizeof(double));
    A((void**)&b->d_wf, wfoff * sizeof(double));
    A((void**)&b->d_R, woff * sizeof(double));
    A((void**)&b->d_bnd, bndoff * sizeof(double));
    A((void**)&b->d_wa, woff * sizeof(double));
    A((void**)&b->d_wb, woff * sizeof(double));
    A((void**)&b->d_dt, P * sizeof(double));
    A((void**)&b->d_t, P * sizeof(double));
    A((void**)&b->d_dtbits, P * sizeof(unsigned long long));
    A((void**)&b->d_flags, sizeof(DevFlags));
    A((void**)&b->d_counters, NCOUNTERS * sizeof(unsigned));
    A((void**)&b->d_done, (size_t)NPH * P * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_probs, b->probs.data(), P * sizeof(ProbDesc), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_nbr, nbr, eoff * 4 * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_h, h, eoff * 2 * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && bcoff > 0) e = cudaMemcpy(b->d_bc, bc, bcoff * 4 * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->d_flags, 0, sizeof(DevFlags));
    if (e == cudaSuccess) e = cudaMemset(b->d_t, 0, P * sizeof(double));
    if (e == cudaSuccess) e = upload_items(b, make_items(b->probs, FR_CHUNK), &b->d_fr_items, &b->n_fr_items);
    if (e == cudaSuccess) {
        cudaFuncSetAttribute(k_batch_stage, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(LimUnion<>));
        e = set_bounds_shape(b, 1, 16, max_bounds_blocks(1));
    }
    if (e != cudaSuccess) {
        kbl_batch_destroy(b);
        return e == cudaErrorMemoryAllocation ? KBL_ENOMEM : KBL_ECUDA;
    }
    *out = b;
    return KBL_OK;
}

kbl_status kbl_batch_destroy(kbl_batch* b)
{
    if (!b) return KBL_EINVAL;
    drop_graph(b);
    drop_groups(b);
    if (b->d_whost) cudaFree(b->d_whost);
    if (b->d_gcounters) cudaFree(b->d_gcounters);
    if (b->s_h2d) cudaStreamDestroy(b->s_h2d);
    if (b->s_d2h) cudaStreamDestroy(b->s_d2h);
    if (b->tb0) cudaEventDestroy(b->tb0);
    if (b->tb1) cudaEventDestroy(b->tb1);
    if (b->d_cnt) cudaFree(b->d_cnt);
    if (b->d_done) cudaFree(b->d_done);
    void* ptrs[] = {b->d_probs, b->d_nbr, b->d_h, b->d_bc, b->d_wf, b->d_R, b->d_bnd, b->d_wa, b->d_wb, b->d_dt,
                    b->d_t, b->d_dtbits, b->d_flags, b->d_counters, b->d_fr_items, b->d_b_items};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    delete b;
    return KBL_OK;
}

const char* kbl_batch_last_error(const kbl_batch* b) { return b ? b->err.c_str() : "null batch"; }
int64_t kbl_batch_launch_count(const kbl_batch* b) { return b ? b->launches : -1; }

kbl_status kbl_batch_layout(const kbl_batch* b, int64_t* so, int64_t* eo)
{
    if (!b || !so || !eo) return KBL_EINVAL;
    for (int i = 0; i < b->P; i++) {
        so[i] = b->probs[i].woff;
        eo[i] = b->probs[i].eoff;
    }
    so[b->P] = b->W_total;
    eo[b->P] = b->E_total;
    return KBL_OK;
}

kbl_status kbl_batch_nodes(const kbl_batch* b, int p, double* out, int n)
{
    if (!b || !out || p < 1 || p > PMAX_B || n < p + 1) return KBL_EINVAL;
    for (int i = 0; i <= p; i++) out[i] = b->ops.o[p].x[i];
    return KBL_OK;
}

kbl_status kbl_batch_step(kbl_batch* b, double* w, double cfl)
{
    if (!b || !w || !(cfl > 0.0)) return bfail(b, KBL_EINVAL, "bad argument");
    if (!(b->graph && b->graph_w == w && b->graph_cfl == cfl)) {
        drop_graph(b);
        int n = 0;
        const cudaError_t e = capture_step(b, w, cfl, all_items(b), &b->graph, &n);
        if (e != cudaSuccess) return bfail(b, KBL_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
        b->graph_w = w;
        b->graph_cfl = cfl;
        b->graph_kernels = n;
    }
    cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
    if (e != cudaSuccess) return bfail(b, KBL_ECUDA, cudaGetErrorString(e));
    b->launches += b->graph_kernels;
    return KBL_OK;
}

// Groups of consecutive problems of roughly equal state size for kbl_batch_run_host, with their
// own work items (bounds items at the current chunk size) and events.
cudaError_t build_groups(kbl_batch* b)
{
    if (!b->groups.empty() && b->groups[0].chunk == b->chunk) return cudaSuccess;
    drop_groups(b);
    const int G = std::min(b->P, KBL_BATCH_HOST_GROUPS);
    int p0 = 0;
    for (int g = 0; g < G; g++) {
        // end of group g: the first problem whose state ends at or past (g + 1) / G of the total
        int p1 = p0 + 1;
        const double target = (double)b->W_total * (g + 1) / G;
        while (p1 < b->P && (double)(b->probs[p1 - 1].woff + 4LL * b->probs[p1 - 1].E * (b->probs[p1 - 1].p + 1) *
                                               (b->probs[p1 - 1].p + 1)) < target)
            p1++;
        if (g == G - 1) p1 = b->P;
        p1 = std::min(p1, b->P - (G - 1 - g));   // leave a problem for every later group
        kbl_batch::Group gr;
        gr.p0 = p0;
        gr.p1 = p1;
        gr.chunk = b->chunk;
        cudaError_t e = upload_items(b, make_items(b->probs, FR_CHUNK, p0, p1), &gr.fr, &gr.n_fr);
        if (e == cudaSuccess) e = upload_items(b, make_items(b->probs, b->chunk, p0, p1), &gr.bi, &gr.n_bi);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&gr.h2d, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&gr.done, cudaEventDisableTiming);
        b->groups.push_back(gr);
        if (e != cudaSuccess) {
            drop_groups(b);
            return e;
        }
        p0 = p1;
    }
    return cudaSuccess;
}

kbl_status kbl_batch_run_host(kbl_batch* b, const double* win, double* wout, int n_steps, double cfl)
{
    if (!b) return KBL_EINVAL;
    if (!win || !wout || n_steps < 0 || !(cfl > 0.0)) return bfail(b, KBL_EINVAL, "bad argument");
    cudaError_t e = cudaSuccess;
    if (!b->d_whost) e = cudaMalloc((void**)&b->d_whost, std::max<long long>(b->W_total, 2) * sizeof(double));
    if (e == cudaSuccess && !b->d_gcounters)
        e = cudaMalloc((void**)&b->d_gcounters, (size_t)NCOUNTERS * KBL_BATCH_HOST_GROUPS * sizeof(unsigned));
    if (e == cudaSuccess && !b->s_h2d) e = cudaStreamCreateWithFlags(&b->s_h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess && !b->s_d2h) e = cudaStreamCreateWithFlags(&b->s_d2h, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = build_groups(b);
    if (e != cudaSuccess) return bfail(b, e == cudaErrorMemoryAllocation ? KBL_ENOMEM : KBL_ECUDA, cudaGetErrorString(e));
    // the copies wait for whatever the caller queued on the batch's stream before this call
    cudaEvent_t start = nullptr;
    if ((e = cudaEventCreateWithFlags(&start, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventRecord(start, b->stream)) != cudaSuccess || (e = cudaStreamWaitEvent(b->s_h2d, start, 0)) != cudaSuccess) {
        if (start) cudaEventDestroy(start);
        return bfail(b, KBL_ECUDA, cudaGetErrorString(e));
    }
    cudaEventDestroy(start);
    const int G = (int)b->groups.size();
    for (int g = 0; g < G && e == cudaSuccess; g++) {
        auto& gr = b->groups[g];
        const long long a = b->probs[gr.p0].woff;
        const long long z = gr.p1 < b->P ? b->probs[gr.p1].woff : b->W_total;
        e = cudaMemcpyAsync(b->d_whost + a, win + a, (size_t)(z - a) * sizeof(double), cudaMemcpyHostToDevice, b->s_h2d);
        if (e == cudaSuccess) e = cudaEventRecord(gr.h2d, b->s_h2d);
    }
    for (int g = 0; g < G && e == cudaSuccess; g++) {
        auto& gr = b->groups[g];
        if (!(gr.graph && gr.cfl == cfl)) {
            if (gr.graph) cudaGraphExecDestroy(gr.graph);
            unsigned* cnt = b->d_gcounters + (size_t)NCOUNTERS * g;
            e = capture_step(b, b->d_whost, cfl, {gr.fr, gr.n_fr, gr.bi, gr.n_bi, cnt, gr.p0, gr.p1}, &gr.graph,
                             &gr.kernels);
            gr.cfl = cfl;
            if (e != cudaSuccess) break;
        }
        e = cudaStreamWaitEvent(b->stream, gr.h2d, 0);
        for (int k = 0; k < n_steps && e == cudaSuccess; k++) {
            e = cudaGraphLaunch(gr.graph, b->stream);
            b->launches += gr.kernels;
        }
        if (e == cudaSuccess) e = cudaEventRecord(gr.done, b->stream);
    }
    for (int g = 0; g < G && e == cudaSuccess; g++) {
        auto& gr = b->groups[g];
        const long long a = b->probs[gr.p0].woff;
        const long long z = gr.p1 < b->P ? b->probs[gr.p1].woff : b->W_total;
        e = cudaStreamWaitEvent(b->s_d2h, gr.done, 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(wout + a, b->d_whost + a, (size_t)(z - a) * sizeof(double), cudaMemcpyDeviceToHost,
                                b->s_d2h);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->s_d2h);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return e == cudaSuccess ? KBL_OK : bfail(b, KBL_ECUDA, cudaGetErrorString(e));
}

kbl_status kbl_batch_bounds_ms(kbl_batch* b, double* ms)
{
    if (!b || !ms) return KBL_EINVAL;
    if (!b->tb_valid) return bfail(b, KBL_ESTATE, "no kbl_batch_bounds call yet");
    float f = 0.0f;
    cudaError_t e = cudaEventSynchronize(b->tb1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&f, b->tb0, b->tb1);
    if (e != cudaSuccess) return bfail(b, KBL_ECUDA, cudaGetErrorString(e));
    *ms = f;
    return KBL_OK;
}

// The phases of one batched stage as separate calls (the same persistent kernels the step
// graph runs), for checking a stage against the single-problem calls on identical inputs.
kbl_status kbl_batch_bounds(kbl_batch* b, const double* w, double* bnd)
{
    if (!b || !w || !bnd) return bfail(b, KBL_EINVAL, "null array");
    cudaStream_t s = b->stream;
    cudaMemsetAsync(b->d_counters, 0, NCOUNTERS * sizeof(unsigned), s);
    k_batch_traces<<<grid_of(b, fr_blocks_per_sm((const void*)k_batch_traces, 0)), NTB, 0, s>>>(
        dev_of(b), b->d_fr_items, b->n_fr_items, b->d_counters + 1, b->ops, w, b->d_wf);
    if (!b->tb0) cudaEventCreate(&b->tb0);
    if (!b->tb1) cudaEventCreate(&b->tb1);
    cudaEventRecord(b->tb0, s);
    launch_bounds_phase(b, w, b->d_wf, bnd, b->d_counters + 2, s, b->d_b_items, b->n_b_items);
    cudaEventRecord(b->tb1, s);
    b->tb_valid = true;
    b->launches += 2;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? KBL_OK : bfail(b, KBL_ECUDA, cudaGetErrorString(e));
}

kbl_status kbl_batch_rhs(kbl_batch* b, const double* w, double* R)
{
    if (!b || !w || !R) return bfail(b, KBL_EINVAL, "null array");
    cudaStream_t s = b->stream;
    const BatchDev bd = dev_of(b);
    cudaMemsetAsync(b->d_counters, 0, NCOUNTERS * sizeof(unsigned), s);
    k_batch_traces<<<grid_of(b, fr_blocks_per_sm((const void*)k_batch_traces, 0)), NTB, 0, s>>>(
        bd, b->d_fr_items, b->n_fr_items, b->d_counters + 1, b->ops, w, b->d_wf);
    k_batch_rhs<<<grid_of(b, fr_blocks_per_sm((const void*)k_batch_rhs, 0)), NTB, 0, s>>>(
        bd, b->d_fr_items, b->n_fr_items, b->d_counters + 3, b->ops, b->phys.gamma, b->phys.flux, w, b->d_wf, R);
    b->launches += 2;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? KBL_OK : bfail(b, KBL_ECUDA, cudaGetErrorString(e));
}

kbl_status kbl_batch_stage(kbl_batch* b, int st, const double* wn, const double* ws, const double* R,
                           const double* bnd, const double* dt_dev, double* wout)
{
    if (!b) return KBL_EINVAL;
    if (st < 0 || st > 2) return bfail(b, KBL_EINVAL, "stage must be 0, 1 or 2");
    if (!wn || !ws || !R || !bnd || !dt_dev || !wout) return bfail(b, KBL_EINVAL, "null array");
    cudaStream_t s = b->stream;
    cudaMemsetAsync(b->d_counters, 0, NCOUNTERS * sizeof(unsigned), s);
    k_batch_stage<<<grid_of(b, fr_blocks_per_sm((const void*)k_batch_stage, sizeof(LimUnion<>))), NTB, sizeof(LimUnion<>),
                    s>>>(dev_of(b), b->d_fr_items, b->n_fr_items, b->d_counters + 4, b->ops, b->phys, st, wn, ws, R,
                         bnd, dt_dev, wout, b->d_flags);
    b->launches += 1;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? KBL_OK : bfail(b, KBL_ECUDA, cudaGetErrorString(e));
}

kbl_status kbl_batch_dt(kbl_batch* b, double* dt_host)
{
    if (!b || !dt_host) return KBL_EINVAL;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess) e = cudaMemcpy(dt_host, b->d_dt, b->P * sizeof(double), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? KBL_OK : bfail(b, KBL_ECUDA, cudaGetErrorString(e));
}

kbl_status kbl_batch_autotune(kbl_batch* b, const double* w, double* out_ms, double* out_cmp)
{
    if (!b || !w) return KBL_EINVAL;
    // traces of w once, then time the bounds phase on every eighth work item
    cudaStream_t s = b->stream;
    cudaMemsetAsync(b->d_counters, 0, NCOUNTERS * sizeof(unsigned), s);
    const BatchDev bd = dev_of(b);
    k_batch_traces<<<grid_of(b, fr_blocks_per_sm((const void*)k_batch_traces, 0)), NTB, 0, s>>>(
        bd, b->d_fr_items, b->n_fr_items, b->d_counters + 1, b->ops, w, b->d_wf);
    b->launches++;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best_ms = 1e30, best_cmp = 0.0;
    const int entry[3] = {b->tile, b->chunk, b->blocks_per_sm};
    int best[3] = {entry[0], entry[1], entry[2]};
    const int chunks[] = {4, 16, 64};
    // thread tiles the step's form can run: the fused launch has 128-thread blocks (4x2, 2x4)
    for (int tile = b->fused ? 1 : 0; tile < 3; tile++) {
        const int maxb = max_bounds_blocks(tile);
        const int pers[] = {maxb, std::max(1, (3 * maxb) / 4), std::max(1, maxb / 2)};
        for (int ci = 0; ci < 3; ci++) {
            std::vector<WorkItem> all = make_items(b->probs, chunks[ci]), sample;
            double cmp = 0.0;
            for (size_t i = 0; i < all.size(); i += 8) {
                sample.push_back(all[i]);
                const int n = b->probs[all[i].prob].p + 1;
                cmp += 4.0 * (n * n + 8 * n) * (double)(NX_B * NX_B) * all[i].n;
            }
            WorkItem* d_sample = nullptr;
            int n_sample = 0;
            if (upload_items(b, sample, &d_sample, &n_sample) != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                if (d_sample) cudaFree(d_sample);
                // back to the launch shape the batch had on entry
                set_bounds_shape(b, entry[0], entry[1], entry[2]);
                return bfail(b, KBL_ECUDA, "autotune upload");
            }
            for (int pi = 0; pi < 3; pi++) {
                if (pi > 0 && pers[pi] == pers[pi - 1]) continue;
                b->tile = tile;
                b->blocks_per_sm = pers[pi];
                float ms = 0.f;
                for (int rep = 0; rep < 2; rep++) {   // first run warms up
                    cudaMemsetAsync(b->d_counters + 2, 0, sizeof(unsigned), s);
                    cudaEventRecord(e0, s);
                    launch_bounds_phase(b, w, b->d_wf, b->d_bnd, b->d_counters + 2, s, d_sample, n_sample);
                    cudaEventRecord(e1, s);
                    b->launches++;
                    cudaEventSynchronize(e1);
                    cudaEventElapsedTime(&ms, e0, e1);
                }
                if (ms < best_ms) {
                    best_ms = ms;
                    best_cmp = cmp;
                    best[0] = tile;
                    best[1] = chunks[ci];
                    best[2] = pers[pi];
                }
            }
            cudaFree(d_sample);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaError_t e = set_bounds_shape(b, best[0], best[1], best[2]);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return bfail(b, KBL_ECUDA, cudaGetErrorString(e));
    if (out_ms) *out_ms = best_ms;
    if (out_cmp) *out_cmp = best_cmp;
    return KBL_OK;
}

kbl_status kbl_batch_tuning(const kbl_batch* b, int32_t* out4)
{
    if (!b || !out4) return KBL_EINVAL;
    out4[0] = b->tile;
    out4[1] = b->chunk;
    out4[2] = b->blocks_per_sm;
    out4[3] = b->n_b_items;
    return KBL_OK;
}

kbl_status kbl_batch_check(kbl_batch* b)
{
    if (!b) return KBL_EINVAL;
    DevFlags f;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess) e = cudaMemcpy(&f, b->d_flags, sizeof(f), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(b->d_flags, 0, sizeof(DevFlags));
    if (e != cudaSuccess) return bfail(b, KBL_ECUDA, cudaGetErrorString(e));
    if (f.timeout) return bfail(b, KBL_ETIMEOUT, "a bounded device wait of the fused step gave up");
    if (f.nonphysical) return bfail(b, KBL_ENONPHYSICAL, "non-physical stencil state");
    return KBL_OK;
}

kbl_status kbl_batch_set_form(kbl_batch* b, int fused)
{
    if (!b || (fused != 0 && fused != 1)) return bfail(b, KBL_EINVAL, "form must be 0 (per-phase launches) or 1 (one launch)");
    b->fused = fused;
    drop_graph(b);
    drop_groups(b);
    return KBL_OK;
}

kbl_status kbl_batch_stall_test(kbl_batch* b, int on, int wait_polls)
{
    if (!b || wait_polls < 1) return KBL_EINVAL;
    b->stall_test = on ? 1 : 0;
    b->wait_polls = wait_polls;
    drop_graph(b);
    drop_groups(b);
    return KBL_OK;
}

}  // extern "C"
