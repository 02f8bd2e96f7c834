// kbl_tri_bounds.cu -- kinetic bounds of triangle stencils gathered inside the bounds kernel.
//
// The stencil of a triangle (Sec. 5) is its ns solution values w[e][0..ns-1], its nfp flux-point
// values wf[e][0..nfp-1] and the exterior value at each flux point: the neighbour's flux-point
// value at the same place (edge g of the neighbour, its point p - k, the edge running the other
// way) or the boundary state.  Gathering it here, straight from w and wf, spares the triangle
// step the stencil array S (written by one kernel, read by the next); the bounds code is the
// explicit-stencil kernels' (bounds2d_f32_core, bounds2d_f64_core), padded by repeating the
// last state (neither the envelopes nor the velocity box change).
#include "kbl_bounds64_body.cuh"

namespace {

using namespace kbl_dev;

struct TriGather {
    const double* w;
    const double* wf;
    const int* nbr;
    const int* nbr_edge;
    const double* bc;
    int ns, nfp, p1;
};

template <int NSTC, int NT>
__device__ __forceinline__ void gather_tri(const TriGather& a, int e, double (*sS)[4])
{
    const int nst = a.ns + 2 * a.nfp;
    for (int r = threadIdx.x; r < NSTC; r += NT) {
        const int rr = r < nst ? r : nst - 1;
        const double* src;
        if (rr < a.ns) {
            src = a.w + ((size_t)e * a.ns + rr) * 4;
        } else if (rr < a.ns + a.nfp) {
            src = a.wf + ((size_t)e * a.nfp + (rr - a.ns)) * 4;
        } else {
            const int q = rr - a.ns - a.nfp, f = q / a.p1, k = q - f * a.p1;
            const int nb = a.nbr[e * 3 + f];
            src = nb >= 0 ? a.wf + ((size_t)nb * a.nfp + a.nbr_edge[e * 3 + f] * a.p1 + (a.p1 - 1 - k)) * 4
                          : a.bc + (size_t)(-nb - 1) * 4;
        }
        const double v0 = src[0], v1 = src[1], v2 = src[2], v3 = src[3];
        sS[r][0] = v0;
        sS[r][1] = v1;
        sS[r][2] = v2;
        sS[r][3] = v3;
    }
}

template <int NSTC, int NX, bool PAD>
__global__ void __launch_bounds__(B2f32<NX, 0>::NT, B2f32<NX, 0>::MINB)
k_bounds_tri_f32(TriGather a, int E, Phys ph, double* __restrict__ bnd, DevFlags* flags)
{
    constexpr int NT = B2f32<NX, 0>::NT;
    __shared__ Bounds2dF32SmemS<NSTC, NX, 0> sm;
    const int e = blockIdx.x;
    bounds2d_f32_core<NSTC, NX, 0, PAD>(sm, [&](double (*sS)[4]) { gather_tri<NSTC, NT>(a, e, sS); }, E, e, ph, bnd,
                                        flags);
}

template <int NSTC, int NX>
__global__ void __launch_bounds__(B2f64<NX>::NT, (B2f64<NX>::NT <= 256 ? 4 : 1))
k_bounds_tri_f64(TriGather a, int E, Phys ph, double* __restrict__ bnd, DevFlags* flags)
{
    constexpr int NT = B2f64<NX>::NT;
    const int e = blockIdx.x;
    bounds2d_f64_core<NSTC, NX>([&](double (*sS)[4]) { gather_tri<NSTC, NT>(a, e, sS); }, E, e, ph, bnd, flags);
}

template <int NSTC, int NX>
void run_tri(const kbl_ctx* c, int E, const TriGather& a, double* bnd, cudaStream_t s)
{
    if (c->cfg.precision == KBL_FP32_MIXED) {
        if (c->cfg.nu[0] != NX || c->phys.qwf)
            k_bounds_tri_f32<NSTC, NX, true><<<E, B2f32<NX, 0>::NT, 0, s>>>(a, E, c->phys, bnd, c->d_flags);
        else
            k_bounds_tri_f32<NSTC, NX, false><<<E, B2f32<NX, 0>::NT, 0, s>>>(a, E, c->phys, bnd, c->d_flags);
    } else {
        k_bounds_tri_f64<NSTC, NX><<<E, B2f64<NX>::NT, 0, s>>>(a, E, c->phys, bnd, c->d_flags);
    }
}

template <int NSTC>
int run_tri_nx(const kbl_ctx* c, int E, const TriGather& a, double* bnd, cudaStream_t s)
{
    switch (kbl_tile_nx(c->cfg.nu[0])) {
        case 8: run_tri<NSTC, 8>(c, E, a, bnd, s); return 1;
        case 16: run_tri<NSTC, 16>(c, E, a, bnd, s); return 1;
        case 32: run_tri<NSTC, 32>(c, E, a, bnd, s); return 1;
        case 64: run_tri<NSTC, 64>(c, E, a, bnd, s); return 1;
    }
    return -1;
}

}  // namespace

int launch_bounds_tri(const kbl_ctx* c, int E, int p, const double* w, const double* wf, const int* nbr,
                      const int* nbr_edge, const double* bc, double* bnd, cudaStream_t s)
{
    if (E == 0) return 0;
    if (c->cfg.dim != 2 || p < 1 || p > 2) return -1;
    TriGather a;
    a.w = w;
    a.wf = wf;
    a.nbr = nbr;
    a.nbr_edge = nbr_edge;
    a.bc = bc;
    a.p1 = p + 1;
    a.ns = (p + 1) * (p + 2) / 2;
    a.nfp = 3 * (p + 1);
    return p == 1 ? run_tri_nx<16>(c, E, a, bnd, s) : run_tri_nx<24>(c, E, a, bnd, s);   // 15 and 24 states
}
