// kbl_stencil.cu -- kinetic bounds of explicit per-element stencils.
//
// Eq. 29-46 take any set of states: the bounds of an element follow from the Maxwellians
// of its stencil whatever element family produced them.  These kernels run the FR path's
// bounds code (bounds2d_f32_core, bounds2d_f64_core) on stencils the caller assembles --
// for triangles with their own solution and face points, or any unstructured mesh whose
// traces live outside this library -- read from S[E][n_states][4].  A stencil shorter than
// the compiled capacity (16, 24, 32, 48 or 64 states) repeats its last state, which changes
// neither the envelopes (a min or max over a repeated value) nor the velocity box.
#include "kbl_bounds64_body.cuh"

namespace {

using namespace kbl_dev;

// Copy the stencil of element e, padded to NSTC states with its last state.
template <int NSTC, int NT>
__device__ __forceinline__ void gather_explicit(const double* __restrict__ S, int nst, int e, double (*sS)[4])
{
    for (int r = threadIdx.x; r < NSTC; r += NT) {
        const double* src = S + ((size_t)e * nst + (r < nst ? r : nst - 1)) * 4;
        const double v0 = src[0], v1 = src[1], v2 = src[2], v3 = src[3];
        sS[r][0] = v0;
        sS[r][1] = v1;
        sS[r][2] = v2;
        sS[r][3] = v3;
    }
}

template <int NSTC, int NX, bool PAD>
__global__ void __launch_bounds__(B2f32<NX, 0>::NT, B2f32<NX, 0>::MINB)
k_bounds_stencil_f32(const double* __restrict__ S, int nst, int E, Phys ph, double* __restrict__ bnd,
                     DevFlags* flags)
{
    constexpr int NT = B2f32<NX, 0>::NT;
    __shared__ Bounds2dF32SmemS<NSTC, NX, 0> sm;
    const int e = blockIdx.x;
    bounds2d_f32_core<NSTC, NX, 0, PAD>(sm, [&](double (*sS)[4]) { gather_explicit<NSTC, NT>(S, nst, e, sS); }, E,
                                        e, ph, bnd, flags);
}

template <int NSTC, int NX>
__global__ void __launch_bounds__(B2f64<NX>::NT, (B2f64<NX>::NT <= 256 ? 4 : 1))
k_bounds_stencil_f64(const double* __restrict__ S, int nst, int E, Phys ph, double* __restrict__ bnd,
                     DevFlags* flags)
{
    constexpr int NT = B2f64<NX>::NT;
    const int e = blockIdx.x;
    bounds2d_f64_core<NSTC, NX>([&](double (*sS)[4]) { gather_explicit<NSTC, NT>(S, nst, e, sS); }, E, e, ph, bnd,
                                flags);
}

template <int NSTC, int NX>
int run_stencil(const kbl_ctx* c, int E, int nst, const double* S, double* bnd, cudaStream_t s)
{
    if (c->cfg.precision == KBL_FP32_MIXED) {
        if (c->cfg.nu[0] != NX || c->phys.qwf)
            k_bounds_stencil_f32<NSTC, NX, true><<<E, B2f32<NX, 0>::NT, 0, s>>>(S, nst, E, c->phys, bnd, c->d_flags);
        else
            k_bounds_stencil_f32<NSTC, NX, false><<<E, B2f32<NX, 0>::NT, 0, s>>>(S, nst, E, c->phys, bnd, c->d_flags);
    } else {
        k_bounds_stencil_f64<NSTC, NX><<<E, B2f64<NX>::NT, 0, s>>>(S, nst, E, c->phys, bnd, c->d_flags);
    }
    return 1;
}

template <int NSTC>
int run_stencil_nx(const kbl_ctx* c, int E, int nst, const double* S, double* bnd, cudaStream_t s)
{
    switch (kbl_tile_nx(c->cfg.nu[0])) {
        case 8: return run_stencil<NSTC, 8>(c, E, nst, S, bnd, s);
        case 16: return run_stencil<NSTC, 16>(c, E, nst, S, bnd, s);
        case 32: return run_stencil<NSTC, 32>(c, E, nst, S, bnd, s);
        case 64: return run_stencil<NSTC, 64>(c, E, nst, S, bnd, s);
    }
    return -1;
}

}  // namespace

int launch_bounds_stencil(const kbl_ctx* c, int E, int nst, const double* S, double* bnd, cudaStream_t s)
{
    if (E == 0) return 0;
    if (c->cfg.dim != 2 || nst < 1 || nst > 64) return -1;
    if (nst <= 16) return run_stencil_nx<16>(c, E, nst, S, bnd, s);
    if (nst <= 24) return run_stencil_nx<24>(c, E, nst, S, bnd, s);   // a P2 triangle's stencil
    if (nst <= 32) return run_stencil_nx<32>(c, E, nst, S, bnd, s);
    if (nst <= 48) return run_stencil_nx<48>(c, E, nst, S, bnd, s);
    return run_stencil_nx<64>(c, E, nst, S, bnd, s);
}
