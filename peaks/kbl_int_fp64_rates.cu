// kbl_int_fp64_rates.cu -- measures the rates of the integer and FP64 operations that the
// FR, limiter and bounds kernels spend outside their FP32 arithmetic: 64-bit index
// arithmetic (the widening multiply-add of an element offset, a full 64-bit multiply, a
// 64-bit add), 32-bit multiply-add, FP64 fused multiply-add, and the FP64 -> FP32
// conversion.  On GB300 the FP64 pipe runs at a small fraction of the FP32 rate, so an
// operation that issues to it costs as much as FP64 arithmetic.
//
// Register-only kernels (8 independent chains per thread, 8 blocks of 256 threads per SM),
// one inline-PTX instruction per chain step so that the compiler cannot merge or drop them.
// Each block records its SM and its start and end in that SM's cycle counter (clock64); an
// SM's rate is the work of its blocks over the span from its first start to its last end.
//
// Build: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o kbl_int_fp64_rates kbl_int_fp64_rates.cu
// Run:   ./kbl_int_fp64_rates
#include <cstdio>

#include <cuda_runtime.h>

namespace {

constexpr int CHAINS = 8, THREADS = 256, BLOCKS_PER_SM = 8;

// KIND: 0 mad.wide.u32 (u64 = u32 * u32 + u64), 1 mul.lo.u64 by a loop-carried factor,
// 2 add.u64, 3 mad.lo.u32, 4 fma.rn.f64, 5 cvt.rn.f32.f64 of a loop-invariant value, 6 shl.b32 +
// lop3 (a bit-field step of the FP32 truncation), 7 cvt.rn.f32.f64 of a changing value (its
// input moves by a 64-bit integer add), 8 cvt.f64.f32 (its result folded in by a 64-bit xor),
// 9 add.rn.f64, 10 setp.lt.f64 + selp (an FP64 comparison), 11 div.rn.f32, 12 sqrt.rn.f32
template <int KIND>
__global__ void __launch_bounds__(THREADS) k_rate(unsigned long long* out, long long* stamps, int iters, unsigned seed)
{
    __syncthreads();
    const long long t0 = clock64();
    unsigned long long u[CHAINS];
    unsigned a[CHAINS];
    double d[CHAINS];
    float f[CHAINS];
#pragma unroll
    for (int i = 0; i < CHAINS; i++) {
        a[i] = seed + threadIdx.x * 7u + (unsigned)i;
        u[i] = (unsigned long long)a[i] * 3u + 1u;
        d[i] = 1.0 + 1e-3 * (double)a[i];
        f[i] = 1.0f + 1e-3f * (float)a[i];
        if (KIND == 7) u[i] = (unsigned long long)__double_as_longlong(d[i]);
    }
    const unsigned k32 = 0x9e3779b1u;
    const unsigned long long k64 = 0x9e3779b97f4a7c15ull;
    const double dk = 1.0000000001, dc = 1e-12;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int i = 0; i < CHAINS; i++) {
            if (KIND == 0) {
                asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(u[i]) : "r"((unsigned)u[i]), "r"(k32));
            } else if (KIND == 1) {
                asm volatile("mul.lo.u64 %0, %0, %1;" : "+l"(u[i]) : "l"(u[(i + 1) % CHAINS] | 1ull));
            } else if (KIND == 2) {
                asm volatile("add.u64 %0, %0, %1;" : "+l"(u[i]) : "l"(k64));
            } else if (KIND == 3) {
                asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[i]) : "r"(k32), "r"(k32));
            } else if (KIND == 4) {
                asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(d[i]) : "d"(dk), "d"(dc));
            } else if (KIND == 5) {
                float g;
                asm volatile("cvt.rn.f32.f64 %0, %1;" : "=f"(g) : "d"(d[i]));
                f[i] += g;   // one FP32 add per conversion keeps the result live
                d[i] = d[i] + 0.0;
            } else if (KIND == 6) {
                asm volatile("shl.b32 %0, %0, 3;\n\tlop3.b32 %0, %0, %1, %2, 0x6a;" : "+r"(a[i]) : "r"(k32), "r"(k32 >> 5));
            } else if (KIND == 7) {
                float g;
                double x = __longlong_as_double((long long)u[i]);
                asm volatile("cvt.rn.f32.f64 %0, %1;" : "=f"(g) : "d"(x));
                u[i] += (unsigned long long)__float_as_uint(g) | 1ull;
            } else if (KIND == 8) {
                double x;
                asm volatile("cvt.f64.f32 %0, %1;" : "=d"(x) : "f"(f[i]));
                u[i] ^= (unsigned long long)__double_as_longlong(x);
                f[i] = __uint_as_float((unsigned)u[i] & 0x3f7fffffu);
            } else if (KIND == 9) {
                asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(d[i]) : "d"(dc));
            } else if (KIND == 10) {
                asm volatile("{\n\t.reg .pred q;\n\tsetp.lt.f64 q, %0, %1;\n\tselp.b32 %2, 1, 2, q;\n\t}"
                             : "+d"(d[i]), "+d"(d[(i + 1) % CHAINS]), "+r"(a[i]));
            } else if (KIND == 11) {
                asm volatile("div.rn.f32 %0, %0, %1;" : "+f"(f[i]) : "f"(1.0000001f));
            } else {
                asm volatile("sqrt.rn.f32 %0, %0;" : "+f"(f[i]));
            }
        }
    }
    unsigned long long s = 0;
#pragma unroll
    for (int i = 0; i < CHAINS; i++) s += u[i] + a[i] + (unsigned long long)(d[i] * 1e3) + (unsigned long long)f[i];
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

// PTX instructions counted per chain step (kinds 6 and 10 issue two; kinds 7 and 8 count
// only the conversion, whose helper integer work is measured by kinds 2 and 6)
constexpr int NK = 13;
constexpr double OPS[NK] = {1, 1, 1, 1, 1, 1, 2, 1, 1, 1, 2, 1, 1};
const char* NAMES[NK] = {"mad.wide.u32 (64-bit offset multiply-add)", "mul.lo.u64", "add.u64", "mad.lo.u32",
                         "fma.rn.f64", "cvt.rn.f32.f64 (invariant input)", "shl.b32 + lop3.b32",
                         "cvt.rn.f32.f64 (changing input, + add.u64)", "cvt.f64.f32 (+ xor.b64)", "add.rn.f64",
                         "setp.lt.f64 + selp.b32", "div.rn.f32", "sqrt.rn.f32"};
// fast kinds run more iterations so that every kernel lasts a few milliseconds
constexpr int ITERS[NK] = {8192, 4096, 16384, 16384, 1024, 1024, 16384, 2048, 2048, 1024, 1024, 2048, 2048};

template <int KIND>
void rate(unsigned long long* out, long long* cyc, int sms)
{
    const int blocks = sms * BLOCKS_PER_SM;
    k_rate<KIND><<<blocks, THREADS>>>(out, cyc, ITERS[KIND], 1u);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0);
    k_rate<KIND><<<blocks, THREADS>>>(out, cyc, ITERS[KIND], 2u);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    long long* h = new long long[3 * blocks];
    cudaMemcpy(h, cyc, sizeof(long long) * 3 * blocks, cudaMemcpyDeviceToHost);
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
    const double ops_block = OPS[KIND] * CHAINS * (double)ITERS[KIND] * THREADS;
    double per_clk_sm = 0.0;
    int used = 0;
    for (int i = 0; i < NSM_MAX; i++)
        if (count[i] > 0 && last[i] > first[i]) {
            per_clk_sm += ops_block * count[i] / (double)(last[i] - first[i]);
            used++;
        }
    per_clk_sm /= used;
    printf("%-44s %8.2f lane-instructions/clk/SM  (%.3f ms)\n", NAMES[KIND], per_clk_sm, ms);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
}

}  // namespace

int main()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * BLOCKS_PER_SM;
    unsigned long long* out = nullptr;
    long long* cyc = nullptr;
    if (cudaMalloc(&out, sizeof(unsigned long long) * blocks * THREADS) != cudaSuccess) return 1;
    if (cudaMalloc(&cyc, sizeof(long long) * 3 * blocks) != cudaSuccess) return 1;
    printf("SMs %d\n", sms);
    rate<0>(out, cyc, sms);
    rate<1>(out, cyc, sms);
    rate<2>(out, cyc, sms);
    rate<3>(out, cyc, sms);
    rate<4>(out, cyc, sms);
    rate<5>(out, cyc, sms);
    rate<6>(out, cyc, sms);
    rate<7>(out, cyc, sms);
    rate<8>(out, cyc, sms);
    rate<9>(out, cyc, sms);
    rate<10>(out, cyc, sms);
    rate<11>(out, cyc, sms);
    rate<12>(out, cyc, sms);
    cudaFree(out);
    cudaFree(cyc);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}
