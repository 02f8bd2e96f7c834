// kbl_fr_tc.cu -- the FR residual of the FP32-mixed path with its operator products on the
// 5th-generation tensor cores (tcgen05, accumulators in tensor memory), element tiles staged by
// TMA (cp.async.bulk.tensor).
//
// Sec. 2.3 (FR with the g_DG correction, Sec. 5) writes the residual of element e, component v,
// solution point (i, j) as
//   R = -(2/h_x) [ sum_m D[i][m] Fx(m, j) + g_L'(x_i) (F*_x,0(j) - Fx_-(j)) + g_R'(x_i) (F*_x,1(j) - Fx_+(j)) ]
//       -(2/h_y) [ the same along y ],
// with Fx_-(j) = sum_m l_m(-1) Fx(m, j) the interpolated discontinuous flux at the face point.
// That interpolation is linear in the solution-point fluxes, so it folds into the derivative:
// D'[i][m] = D[i][m] - g_L'(x_i) l_m(-1) - g_R'(x_i) l_m(+1), and the residual of a whole element
// becomes one dense product
//   R[(e, v), n] = sum_k X[(e, v), k] B[k, n],
//   X = [(2/h_x) Fx at the Ns points | (2/h_y) Fy at the Ns points | (2/h_x) F* at the 2N x-face
//        points | (2/h_y) F* at the 2N y-face points],   K = 2 Ns + 4 N,
// with B built once per order on the host (-D' blocks, -g' lifting blocks).  A tile of 32
// elements x 4 components is M = 128 rows; N = Ns padded to 16; K padded to 8.
//
// Precision: the fluxes are FP32 (as in the FP32-mixed residual on CUDA cores); X and B are split
// into TF32 pairs (x = hi + lo) and the product is hi*hi + lo*hi + hi*lo, three tcgen05.mma of
// kind::tf32 per k-step accumulating in FP32 in tensor memory: the dropped lo*lo term and the
// TF32 rounding of lo are 2^-22 of each product, the FP32 level.
//
// Per tile (persistent blocks of 8 warps, 3 per SM): thread 0 arms an mbarrier and issues the TMA
// loads of the state tile (2D map [component][element * points], boxes of 16 elements; elements
// past the mesh read as zeros); meanwhile the threads form the face-point columns of X from the
// traces (own and exterior, read from global memory), then, once the tile has landed, the
// solution-point columns, in shared memory in the K-major no-swizzle layout (8-row x 16-byte core
// matrices; each warp writes whole core matrices, 32 banks); thread 0 issues the MMAs and a
// tcgen05.commit to a second mbarrier; warps w and w + 4 read rows 32 (w % 4) .. of the
// accumulator (columns 0-7 and 8-15) with tcgen05.ld and write R (FP64, exact widening).  The
// next tile's TMA is issued as soon as the current state tile is consumed.  Every wait on an
// mbarrier is bounded: on expiry the block raises the timeout flag, stops taking tiles, waits
// (bounded) for its MMA in flight, frees its tensor memory and returns.
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "kbl_fr_body.cuh"

namespace {

using namespace kbl_dev;

constexpr int TC_EL = 32;         // elements per tile (x 4 components = 128 rows)
constexpr int TC_NT = 256;        // threads per block (8 warps)
constexpr int TC_HALF = 16;       // elements per TMA box
constexpr int TC_TMEM_COLS = 32;  // tensor-memory columns per block (accumulator needs 16)
constexpr int TC_MINB = 3;        // resident blocks per SM (shared memory ~71 KB each)

template <int N>
struct TcShape {
    static constexpr int NS = N * N, NFP = 4 * N;
    static constexpr int K = 2 * NS + 4 * N;          // 48 (P3), 30 (P2)
    static constexpr int KP = (K + 7) / 8 * 8;        // multiple of the MMA k-step (8 TF32)
    static constexpr int NG = (NS + 15) / 16 * 16;    // GEMM N (M = 128 needs a multiple of 16)
    static constexpr int KC = KP / 4;                 // 16-byte core matrices along K
    static constexpr int SBO = KC * 128;              // bytes between 8-row groups
    static constexpr int A_BYTES = (128 / 8) * SBO;
    static constexpr int B_BYTES = (NG / 8) * SBO;
    static constexpr int W_BYTES = 4 * TC_EL * NS * 8;     // state tile, FP64 (TMA)
    // dynamic shared memory layout (offsets from a 1024-byte aligned base)
    static constexpr int OFF_W = 0;
    static constexpr int OFF_AH = (OFF_W + W_BYTES + 1023) / 1024 * 1024;
    static constexpr int OFF_AL = OFF_AH + A_BYTES;
    static constexpr int OFF_BH = OFF_AL + A_BYTES;
    static constexpr int OFF_BL = OFF_BH + B_BYTES;
    static constexpr int OFF_H = OFF_BL + B_BYTES;                       // float2 [32]
    static constexpr int OFF_BAR = OFF_H + TC_EL * 8;                    // 2 mbarriers
    static constexpr int OFF_MISC = OFF_BAR + 16;                        // tmem address, status
    static constexpr int BYTES = OFF_MISC + 16 + 1024;                   // + alignment slack
    // work decomposition: a warp covers 8 elements x 4 points (one 8 x 4 core-matrix block of X
    // per component, so its shared-memory writes hit 32 different banks)
    static constexpr int NODE_GROUPS = (NS + 3) / 4, FACE_GROUPS = (NFP + 3) / 4;
};

// Byte offset of element (row, k) of a TF32 operand in the K-major no-swizzle canonical layout:
// 8 x 4 core matrices of 128 contiguous bytes, K-adjacent core matrices 128 bytes apart (LBO),
// 8-row groups kc * 128 bytes apart (SBO).
__host__ __device__ constexpr int tc_off(int row, int k, int kc)
{
    return (row >> 3) * kc * 128 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

// ---- inline PTX: shared-memory addresses, mbarriers, TMA, tcgen05 -------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: about a second at most, then false
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity)
{
    for (int it = 0; it < (1 << 22); it++) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it > 64) __nanosleep(256);
    }
    return false;
}
__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap* map, int x, int y, unsigned bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// K-major, no-swizzle shared-memory matrix descriptor (tcgen05): start address, leading byte
// offset (K-adjacent core matrices), stride byte offset (8-row groups), descriptor version 1.
__device__ __forceinline__ unsigned long long tc_desc(unsigned addr, unsigned lbo, unsigned sbo)
{
    unsigned long long d = 0;
    d |= (unsigned long long)((addr & 0x3FFFFu) >> 4);
    d |= (unsigned long long)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (unsigned long long)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;   // version
    return d;          // base offset 0, relative LBO, layout type 0 (no swizzle)
}
// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major, M x N.
__host__ __device__ constexpr unsigned tc_idesc(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(unsigned tmem, unsigned long long a, unsigned long long b, unsigned idesc,
                                       unsigned accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void tc_commit(unsigned bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_ld8(unsigned taddr, float (&v)[8])
{
    unsigned r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; i++) v[i] = __uint_as_float(r[i]);
}
// TF32 split of an FP32 value: hi = x rounded to TF32, lo = (x - hi) rounded to TF32.
__device__ __forceinline__ void tf32_split(float x, unsigned& hi, unsigned& lo)
{
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(x));
    const float r = x - __uint_as_float(hi);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(lo) : "f"(r));
}

struct TcArgs {
    const double* wf;    // traces [4][E][Nfp] (exterior values are read from here)
    MeshDev m;
    const float* op;     // B_hi then B_lo in the canonical layout (2 B_BYTES), device
    double gamma;
    int flux;
    double* R;
    DevFlags* flags;
};

template <int N>
__global__ void __launch_bounds__(TC_NT, TC_MINB)
k_rhs_tc(const __grid_constant__ CUtensorMap map_w, TcArgs a)
{
    using SH = TcShape<N>;
    constexpr int NS = SH::NS, NFP = SH::NFP, KP = SH::KP, KC = SH::KC, NG = SH::NG;
    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char* sm = (unsigned char*)(((size_t)smraw + 1023) & ~(size_t)1023);
    const double* sW = (const double*)(sm + SH::OFF_W);
    unsigned* sAh = (unsigned*)(sm + SH::OFF_AH);
    unsigned* sAl = (unsigned*)(sm + SH::OFF_AL);
    float2* sH = (float2*)(sm + SH::OFF_H);
    const unsigned bar_tma = smem_u32(sm + SH::OFF_BAR), bar_mma = bar_tma + 8;
    unsigned* s_misc = (unsigned*)(sm + SH::OFF_MISC);   // [0] tmem address, [1] status
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int E = a.m.E;
    const int ntiles = (E + TC_EL - 1) / TC_EL;
    constexpr unsigned TX_BYTES = (unsigned)SH::W_BYTES;
    constexpr int NW = TC_NT / 32;

    // set-up: operator B into shared memory, barriers, tensor memory
    {
        const unsigned* src = (const unsigned*)a.op;
        unsigned* dst = (unsigned*)(sm + SH::OFF_BH);
        for (int i = tid; i < 2 * SH::B_BYTES / 4; i += TC_NT) dst[i] = src[i];
    }
    if (tid == 0) {
        mbar_init(bar_tma, 1);
        mbar_init(bar_mma, 1);
        s_misc[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_misc)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = s_misc[0];
    const float gamma = from_f64<float>(a.gamma), gm1 = gamma - 1.0f;

    int tile = blockIdx.x;
    if (tid == 0 && tile < ntiles) {
        mbar_expect_tx(bar_tma, TX_BYTES);
        for (int hf = 0; hf < 2; hf++)
            tma_load_2d(smem_u32(sW) + hf * (SH::W_BYTES / 2), &map_w, (tile * TC_EL + hf * TC_HALF) * NS, 0, bar_tma);
    }
    // what a failed wait may leave in flight: the MMA of tile `it` (parity it & 1), the TMA of
    // the following tile (parity (it + 1) & 1)
    bool mma_in_flight = false, tma_next = false;
    unsigned it = 0;
    for (; tile < ntiles; it++, tile += gridDim.x) {
        const int e0 = tile * TC_EL;
        const int nel = min(TC_EL, E - e0);
        if (tid < TC_EL) {   // the 2/h factors
            float2 s = make_float2(0.f, 0.f);
            if (tid < nel) {
                s.x = 2.0f / from_f64<float>(a.m.h[(size_t)(e0 + tid) * 2 + 0]);
                s.y = 2.0f / from_f64<float>(a.m.h[(size_t)(e0 + tid) * 2 + 1]);
            }
            sH[tid] = s;
        }
        // X, face points first (their traces come from global memory, as the state tile lands):
        // common fluxes scaled by 2/h of their axis
        for (int wq = warp; wq < 4 * SH::FACE_GROUPS; wq += NW) {
            const int el = ((wq & 3) << 3) | (lane >> 2), fp = ((wq >> 2) << 2) | (lane & 3);
            if (fp >= NFP) continue;
            float Fc[4] = {0.f, 0.f, 0.f, 0.f};
            if (el < nel) {
                const int e = e0 + el;
                const int f = fp / N, dir = f >> 1, side = f & 1;
                float qi[4], qe[4];
#pragma unroll
                for (int v = 0; v < 4; v++) {
                    qi[v] = from_f64<float>(a.wf[((size_t)v * E + e) * NFP + fp]);
                    qe[v] = from_f64<float>(kbl_exterior<2, N>(a.wf, a.m, e, fp, v));
                }
                const float* ql = side ? qi : qe;
                const float* qr = side ? qe : qi;
                if (a.flux == 1) kbl_hllc<2, float>(ql, qr, dir, gamma, Fc);
                else if (a.flux == 2) kbl_hll<2, float>(ql, qr, dir, gamma, Fc);
                else kbl_rusanov<2, float>(ql, qr, dir, gamma, Fc);
                const float s = dir ? 2.0f / from_f64<float>(a.m.h[(size_t)e * 2 + 1])
                                    : 2.0f / from_f64<float>(a.m.h[(size_t)e * 2 + 0]);
#pragma unroll
                for (int v = 0; v < 4; v++) Fc[v] *= s;
            }
#pragma unroll
            for (int v = 0; v < 4; v++) {
                const int row = v * TC_EL + el;
                unsigned hi, lo;
                tf32_split(Fc[v], hi, lo);
                sAh[tc_off(row, 2 * NS + fp, KC) / 4] = hi;
                sAl[tc_off(row, 2 * NS + fp, KC) / 4] = lo;
            }
        }
        if (SH::K < KP) {   // zero padding columns of K
            for (int idx = tid; idx < 128 * (KP - SH::K); idx += TC_NT) {
                const int row = idx / (KP - SH::K), k = SH::K + idx % (KP - SH::K);
                sAh[tc_off(row, k, KC) / 4] = 0u;
                sAl[tc_off(row, k, KC) / 4] = 0u;
            }
        }
        // the tile's state
        if (tid == 0 && !mbar_wait_bounded(bar_tma, it & 1)) s_misc[1] = 1;
        __syncthreads();
        if (s_misc[1]) break;
        // X: fluxes at the solution points, scaled by 2/h
        for (int wq = warp; wq < 4 * SH::NODE_GROUPS; wq += NW) {
            const int el = ((wq & 3) << 3) | (lane >> 2), nd = ((wq >> 2) << 2) | (lane & 3);
            if (nd >= NS) continue;
            float Fx[4] = {0.f, 0.f, 0.f, 0.f}, Fy[4] = {0.f, 0.f, 0.f, 0.f};
            if (el < nel) {
                const double* src = sW + (el / TC_HALF) * (4 * TC_HALF * NS) + (el % TC_HALF) * NS + nd;
                float q[4];
#pragma unroll
                for (int v = 0; v < 4; v++) q[v] = from_f64<float>(src[v * TC_HALF * NS]);
                kbl_flux<2, float>(q, 0, gm1, Fx);
                kbl_flux<2, float>(q, 1, gm1, Fy);
                const float2 s = sH[el];
#pragma unroll
                for (int v = 0; v < 4; v++) {
                    Fx[v] *= s.x;
                    Fy[v] *= s.y;
                }
            }
#pragma unroll
            for (int v = 0; v < 4; v++) {
                const int row = v * TC_EL + el;
                unsigned hi, lo;
                tf32_split(Fx[v], hi, lo);
                sAh[tc_off(row, nd, KC) / 4] = hi;
                sAl[tc_off(row, nd, KC) / 4] = lo;
                tf32_split(Fy[v], hi, lo);
                sAh[tc_off(row, NS + nd, KC) / 4] = hi;
                sAl[tc_off(row, NS + nd, KC) / 4] = lo;
            }
        }
        fence_proxy_async();   // X (generic writes) visible to the tensor core (async proxy)
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            // the next tile's TMA may overwrite the state tile now
            const int nt = tile + gridDim.x;
            tma_next = nt < ntiles;
            if (nt < ntiles) {
                mbar_expect_tx(bar_tma, TX_BYTES);
                for (int hf = 0; hf < 2; hf++)
                    tma_load_2d(smem_u32(sW) + hf * (SH::W_BYTES / 2), &map_w, (nt * TC_EL + hf * TC_HALF) * NS, 0,
                                bar_tma);
            }
            const unsigned idesc = tc_idesc(128, NG);
            const unsigned ah = smem_u32(sAh), al = smem_u32(sAl);
            const unsigned bh = smem_u32(sm + SH::OFF_BH), bl = smem_u32(sm + SH::OFF_BL);
#pragma unroll
            for (int ks = 0; ks < KP / 8; ks++) {
                const unsigned off = ks * 256;   // two K-adjacent core matrices per k-step
                tc_mma(tmem, tc_desc(ah + off, 128, SH::SBO), tc_desc(bh + off, 128, SH::SBO), idesc, ks > 0);
                tc_mma(tmem, tc_desc(al + off, 128, SH::SBO), tc_desc(bh + off, 128, SH::SBO), idesc, 1);
                tc_mma(tmem, tc_desc(ah + off, 128, SH::SBO), tc_desc(bl + off, 128, SH::SBO), idesc, 1);
            }
            tc_commit(bar_mma);
        }
        mma_in_flight = true;
        if (tid == 0 && !mbar_wait_bounded(bar_mma, it & 1)) s_misc[1] = 2;
        __syncthreads();
        if (s_misc[1]) break;
        mma_in_flight = false;
        tc_fence_after();
        // epilogue: warp w holds rows 32 (w % 4) .. + 31 = component w % 4 of the tile's 32
        // elements, columns 8 (w / 4) .. + 7
        float acc[8];
        const int cq = warp >> 2;
        tc_ld8(tmem + ((unsigned)((warp & 3) * 32) << 16) + (unsigned)(cq * 8), acc);
        if (lane < nel) {
            double* dst = a.R + ((size_t)(warp & 3) * E + e0 + lane) * NS;
#pragma unroll
            for (int n = 0; n < 8; n++)
                if (cq * 8 + n < NS) dst[cq * 8 + n] = to_f64<float>(acc[n]);
        }
        tc_fence_before();
        __syncthreads();   // accumulator and X free for the next tile
    }
    if (s_misc[1]) {
        // a wait ran out: report it, then let whatever this block still has in flight finish
        // (bounded) before its shared and tensor memory are released
        if (tid == 0) {
            atomicOr(&a.flags->timeout, 1);
            if (s_misc[1] == 2 && mma_in_flight) mbar_wait_bounded(bar_mma, it & 1);
            if (s_misc[1] == 2 && tma_next) mbar_wait_bounded(bar_tma, (it + 1) & 1);
        }
        __syncthreads();
    }
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
}

// ---- host ------------------------------------------------------------------
// TF32 of an FP64 value: round to nearest (ties away) on 10 explicit mantissa bits, as
// cvt.rna.tf32.f32 does after the FP32 rounding.
float tf32_host(double x)
{
    float f = (float)x;
    unsigned u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) {
        u += 0x1000u;
        u &= 0xffffe000u;
    }
    std::memcpy(&f, &u, 4);
    return f;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// 2D map of an array [4][E * pts] of doubles, box [4][16 * pts].
bool make_map(CUtensorMap* map, const double* base, int E, int pts)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)E * pts, 4};
    const cuuint64_t strides[1] = {(cuuint64_t)E * pts * 8};
    const cuuint32_t box[2] = {(cuuint32_t)(TC_HALF * pts), 4};
    const cuuint32_t es[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int N>
int run_rhs_tc(const kbl_ctx* c, const double* w, const double* wf, double* R, cudaStream_t s)
{
    using SH = TcShape<N>;
    if (c->E == 0) return 0;
    // TMA of the state: 16-byte aligned base and row stride (E * Ns * 8 a multiple of 16)
    if (((size_t)w & 15) || ((size_t)c->E * SH::NS * 8) % 16) return -2;
    CUtensorMap mw;
    if (!make_map(&mw, w, c->E, SH::NS)) return -2;
    if (cudaFuncSetAttribute(k_rhs_tc<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, SH::BYTES) != cudaSuccess ||
        cudaFuncSetAttribute(k_rhs_tc<N>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
            cudaSuccess)
        return -2;
    // resident blocks per SM from the device's limits: the occupancy query does not see the
    // shared-memory carveout set above and answers 1.  Registers: __launch_bounds__(TC_NT,
    // TC_MINB); shared memory: the per-SM capacity over the block's share (plus the 1 KB the
    // runtime reserves per block); tensor memory: 512 columns per SM.
    int dev = 0, nsm = 0, smem_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    int per = std::min(TC_MINB, smem_sm / (SH::BYTES + 1024));
    per = std::max(1, std::min(per, 512 / TC_TMEM_COLS));
    const int ntiles = (c->E + TC_EL - 1) / TC_EL;
    const int grid = std::min(ntiles, nsm * per);
    TcArgs a;
    a.wf = wf;
    a.m = mesh_of(c);
    a.op = c->d_tcop;
    a.gamma = c->phys.gamma;
    a.flux = c->phys.flux;
    a.R = R;
    a.flags = c->d_flags;
    k_rhs_tc<N><<<grid, TC_NT, SH::BYTES, s>>>(mw, a);
    return 1;
}

}  // namespace

// The folded residual operator B[k][n] of order p (FP64, K x Ns, row-major; see the top of this
// file), used by the host-side split and by kbl_get_operator.
void kbl_rhs_operator(const FrOps& o, int p, std::vector<double>& B, int& K, int& NS)
{
    const int n = p + 1;
    NS = n * n;
    K = 2 * NS + 4 * n;
    B.assign((size_t)K * NS, 0.0);
    for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) {
            const int t = j * n + i;   // target solution point (i along x, j along y)
            for (int m = 0; m < n; m++) {
                const double dx = o.D[i][m] - o.gl[i] * o.lm[m] - o.gr[i] * o.lp[m];
                const double dy = o.D[j][m] - o.gl[j] * o.lm[m] - o.gr[j] * o.lp[m];
                B[(size_t)(j * n + m) * NS + t] = -dx;        // Fx at (m, j)
                B[(size_t)(NS + m * n + i) * NS + t] = -dy;   // Fy at (i, m)
            }
            B[(size_t)(2 * NS + 0 * n + j) * NS + t] = -o.gl[i];   // F* at face 0 (-x), point j
            B[(size_t)(2 * NS + 1 * n + j) * NS + t] = -o.gr[i];   // face 1 (+x)
            B[(size_t)(2 * NS + 2 * n + i) * NS + t] = -o.gl[j];   // face 2 (-y), point i
            B[(size_t)(2 * NS + 3 * n + i) * NS + t] = -o.gr[j];   // face 3 (+y)
        }
}

// Device copy of the split operator of order p in the kernel's shared-memory layout, or nullptr
// when the tensor-core residual does not cover the order (then the caller keeps the CUDA-core
// residual).  Returns the allocation (the caller frees it).
float* kbl_rhs_tc_upload(const FrOps& o, int p)
{
    auto build = [&](auto shape) -> float* {
        using SH = decltype(shape);
        std::vector<double> B;
        int K = 0, NS = 0;
        kbl_rhs_operator(o, p, B, K, NS);
        std::vector<float> h(2 * SH::B_BYTES / 4, 0.0f);
        for (int k = 0; k < K; k++)
            for (int t = 0; t < NS; t++) {
                const double b = B[(size_t)k * NS + t];
                const float hi = tf32_host(b);
                const float lo = tf32_host(b - (double)hi);
                h[tc_off(t, k, SH::KC) / 4] = hi;
                h[SH::B_BYTES / 4 + tc_off(t, k, SH::KC) / 4] = lo;
            }
        float* d = nullptr;
        if (cudaMalloc((void**)&d, h.size() * 4) != cudaSuccess) return nullptr;
        if (cudaMemcpy(d, h.data(), h.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaFree(d);
            return nullptr;
        }
        return d;
    };
    if (p == 2) return build(TcShape<3>{});
    if (p == 3) return build(TcShape<4>{});
    return nullptr;
}

// -1: not covered (order, dimension, precision or knob); -2: covered but not launchable for these
// arrays (alignment, tensor map): the caller falls back to the CUDA-core kernel.
int launch_rhs_tc(const kbl_ctx* c, const double* w, const double* wf, double* R, cudaStream_t s)
{
    if (!c->d_tcop || c->rhs_tc == 0 || c->cfg.dim != 2 || c->cfg.precision != KBL_FP32_MIXED) return -1;
    if (c->cfg.p == 2) return run_rhs_tc<3>(c, w, wf, R, s);
    if (c->cfg.p == 3) return run_rhs_tc<4>(c, w, wf, R, s);
    return -1;
}
