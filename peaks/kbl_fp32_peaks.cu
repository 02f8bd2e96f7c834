// kbl_fp32_peaks.cu -- measures the FP32 instruction rates that bound the kinetic-bounds
// envelope loop on this GPU, and whether multiplies and min/max share one issue budget.
//
// Register-only kernels (8 independent chains per thread, 8 blocks of 256 threads per SM)
// time FMUL, packed FMUL2, two-input FMNMX, three-input FMNMX3 alone, and the envelope
// pattern (two packed products, then four three-input min/max per pair of values).  Each
// block records its SM and its start and end in that SM's cycle counter (clock64); an SM's
// rate is the work of its blocks over the span from its first start to its last end, so
// the rates are per clock whatever the clock was.  The event-timed wall rate and the
// implied mean SM clock are printed beside them.  Multiplies count one operation per product, min/max one per
// comparison.
//
// Build: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o kbl_fp32_peaks kbl_fp32_peaks.cu
// Run:   ./kbl_fp32_peaks
#include <algorithm>
#include <cstdio>
#include <cstdlib>

#include <cuda_runtime.h>

namespace {

constexpr int CHAINS = 8, ITERS = 65536, THREADS = 256, BLOCKS_PER_SM = 8;

__device__ __forceinline__ float mn3(float a, float b, float c)
{
    float r;
    asm volatile("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float mx3(float a, float b, float c)
{
    float r;
    asm volatile("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float mn2(float a, float b)
{
    float r;
    asm volatile("min.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float mx2(float a, float b)
{
    float r;
    asm volatile("max.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// KIND: 0 FMUL, 1 FMUL2, 2 FMNMX, 3 FMNMX3, 4 envelope pattern (2 FMUL2 + 4 FMNMX3),
// 5 the same work with scalar products (4 FMUL + 4 FMNMX3), 6 with two-input min/max
// (2 FMUL2 + 8 FMNMX), 7 half packed, half scalar products (1 FMUL2 + 2 FMUL + 4 FMNMX3)
template <int KIND>
__global__ void __launch_bounds__(THREADS) k_rate(float* out, long long* stamps, float seed)
{
    __syncthreads();
    const long long t0 = clock64();
    float a[CHAINS], b[CHAINS], c[CHAINS], d[CHAINS];
    float2 p[CHAINS];
#pragma unroll
    for (int i = 0; i < CHAINS; i++) {
        a[i] = seed + threadIdx.x * 1e-3f + i;
        b[i] = a[i] * 0.5f;
        c[i] = a[i] + 1.0f;
        d[i] = a[i] - 1.0f;
        p[i] = make_float2(a[i], b[i]);
    }
    const float2 k = make_float2(1.0000001f, 0.9999999f);
    for (int it = 0; it < ITERS; it++) {
#pragma unroll
        for (int i = 0; i < CHAINS; i++) {
            if (KIND == 0) {
                a[i] = a[i] * 1.0000001f;
                b[i] = b[i] * 0.9999999f;
            } else if (KIND == 1) {
                p[i] = mul2(p[i], k);
            } else if (KIND == 2) {
                a[i] = mn2(a[i], b[i]);
                b[i] = mn2(b[i], c[i]);
            } else if (KIND == 3) {
                a[i] = mn3(a[i], b[i], c[i]);
                d[i] = mx3(d[i], b[i], c[i]);
            } else if (KIND == 5) {
                const float gx = p[i].x * 1.0000001f, gy = p[i].y * 0.9999999f;
                const float hx = b[i] * 1.0000001f, hy = c[i] * 0.9999999f;
                a[i] = mn3(a[i], gx, gy);
                d[i] = mx3(d[i], gx, gy);
                b[i] = mn3(b[i], hx, hy);
                c[i] = mx3(c[i], hx, hy);
                p[i] = make_float2(gy, gx);
            } else if (KIND == 6) {
                const float2 g = mul2(p[i], k);
                const float2 h = mul2(make_float2(b[i], c[i]), k);
                a[i] = mn2(mn2(a[i], g.x), g.y);
                d[i] = mx2(mx2(d[i], g.x), g.y);
                b[i] = mn2(mn2(b[i], h.x), h.y);
                c[i] = mx2(mx2(c[i], h.x), h.y);
                p[i] = make_float2(g.y, g.x);
            } else if (KIND == 7) {
                const float2 g = mul2(p[i], k);
                const float hx = b[i] * 1.0000001f, hy = c[i] * 0.9999999f;
                a[i] = mn3(a[i], g.x, g.y);
                d[i] = mx3(d[i], g.x, g.y);
                b[i] = mn3(b[i], hx, hy);
                c[i] = mx3(c[i], hx, hy);
                p[i] = make_float2(g.y, g.x);
            } else {
                const float2 g = mul2(p[i], k);
                const float2 h = mul2(make_float2(b[i], c[i]), k);
                a[i] = mn3(a[i], g.x, g.y);
                d[i] = mx3(d[i], g.x, g.y);
                b[i] = mn3(b[i], h.x, h.y);
                c[i] = mx3(c[i], h.x, h.y);
                p[i] = make_float2(g.y, g.x);
            }
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < CHAINS; i++) s += a[i] + b[i] + c[i] + d[i] + p[i].x + p[i].y;
    out[blockIdx.x * THREADS + threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        stamps[3 * blockIdx.x + 0] = smid;
        stamps[3 * blockIdx.x + 1] = t0;
        stamps[3 * blockIdx.x + 2] = clock64();
    }
}

// lane-operations per thread per iteration of each kind
constexpr double OPS[8] = {2.0 * CHAINS, 2.0 * CHAINS, 2.0 * CHAINS, 4.0 * CHAINS,
                          12.0 * CHAINS, 12.0 * CHAINS, 12.0 * CHAINS, 12.0 * CHAINS};
const char* NAMES[8] = {"FMUL (1 product)", "FMUL2 (2 products)", "FMNMX (1 comparison)",
                        "FMNMX3 (2 comparisons)", "envelope pattern (4 products + 8 comparisons)",
                        "  same, scalar FMUL products", "  same, two-input FMNMX",
                        "  same, half FMUL2 half FMUL"};

template <int KIND>
double rate(float* out, long long* cyc, int sms)
{
    const int blocks = sms * BLOCKS_PER_SM;
    k_rate<KIND><<<blocks, THREADS>>>(out, cyc, 1.0f);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0);
    k_rate<KIND><<<blocks, THREADS>>>(out, cyc, 2.0f);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    long long* h = new long long[3 * blocks];
    cudaMemcpy(h, cyc, sizeof(long long) * 3 * blocks, cudaMemcpyDeviceToHost);
    // per SM: blocks run, first start, last end
    const int NSM_MAX = 1024;
    static long long first[NSM_MAX], last[NSM_MAX];
    static int count[NSM_MAX];
    for (int i = 0; i < NSM_MAX; i++) { first[i] = -1; last[i] = 0; count[i] = 0; }
    for (int b = 0; b < blocks; b++) {
        const int sm = (int)h[3 * b];
        if (sm < 0 || sm >= NSM_MAX) continue;
        if (first[sm] < 0 || h[3 * b + 1] < first[sm]) first[sm] = h[3 * b + 1];
        if (h[3 * b + 2] > last[sm]) last[sm] = h[3 * b + 2];
        count[sm]++;
    }
    delete[] h;
    const double ops_block = OPS[KIND] * ITERS * THREADS;
    double per_clk_sm = 0.0, mean_cycles = 0.0;
    int used = 0;
    for (int i = 0; i < NSM_MAX; i++)
        if (count[i] > 0 && last[i] > first[i]) {
            per_clk_sm += ops_block * count[i] / (double)(last[i] - first[i]);
            mean_cycles += (double)(last[i] - first[i]);
            used++;
        }
    per_clk_sm /= used;
    mean_cycles /= used;
    const double wall = ops_block * blocks / (ms * 1e-3);
    printf("%-48s %7.1f lane-ops/clk/SM  %7.2f T lane-ops/s  (mean SM clock %.0f MHz)\n", NAMES[KIND], per_clk_sm,
           wall * 1e-12, mean_cycles / (ms * 1e-3) * 1e-6);
    return per_clk_sm;
}

}  // namespace

int main()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * BLOCKS_PER_SM;
    float* out = nullptr;
    long long* cyc = nullptr;
    if (cudaMalloc(&out, sizeof(float) * blocks * THREADS) != cudaSuccess) return 1;
    if (cudaMalloc(&cyc, sizeof(long long) * 3 * blocks) != cudaSuccess) return 1;
    printf("SMs %d\n", sms);
    rate<0>(out, cyc, sms);
    const double r1 = rate<1>(out, cyc, sms);
    rate<2>(out, cyc, sms);
    const double r3 = rate<3>(out, cyc, sms);
    const double r4 = rate<4>(out, cyc, sms);
    rate<5>(out, cyc, sms);
    rate<6>(out, cyc, sms);
    rate<7>(out, cyc, sms);
    // separate budgets: the envelope pattern would run at the slower of its two parts alone;
    // one shared budget: its time would be the sum of both
    const double t_sep = std::max(4.0 / r1, 8.0 / r3), t_sum = 4.0 / r1 + 8.0 / r3;
    printf("envelope pattern: %.1f lane-ops/clk/SM; separate budgets would give %.1f, one shared budget %.1f\n",
           r4, 12.0 / t_sep, 12.0 / t_sum);
    cudaFree(out);
    cudaFree(cyc);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}
