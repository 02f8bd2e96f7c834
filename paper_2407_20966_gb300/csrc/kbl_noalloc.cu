// kbl_noalloc.cu -- kbl_bounds_noalloc: the element bounds for callers that must
// not allocate device memory.
//
// The bounds need the face traces of the solution as scratch.  kbl_bounds gets
// them from a context whose scratch kbl_mesh_upload allocated; this entry point
// instead keeps them in a file-scope device array of fixed size, so it needs
// no context, no cudaMalloc and no host allocation.  The kernels are the same
// traces and bounds kernels that kbl_traces / kbl_bounds launch.
#include <mutex>

#include "kbl_internal.cuh"

// Scratch for the face traces: 1 Mi doubles (8 MiB), i.e. n_elem * (d+2) * Nfp
// values at most (16384 two-dimensional P3 elements).  Every GPU that loads the
// library holds this array until the process exits.
#define KBL_NOALLOC_MAX_TRACE_VALUES (1u << 20)
static __device__ __align__(256) double g_noalloc_traces[KBL_NOALLOC_MAX_TRACE_VALUES];
static __device__ __align__(256) DevFlags g_noalloc_flags;

namespace {

constexpr int MAX_DEVICES = 64;

struct SymbolAddrs {
    bool ready = false;
    double* traces = nullptr;
    DevFlags* flags = nullptr;
};

SymbolAddrs g_addrs[MAX_DEVICES];
std::mutex g_addrs_lock;

// Device addresses of the scratch arrays for the current device, looked up
// once per device (host code must not use the symbols' host-side names).
cudaError_t symbol_addrs(SymbolAddrs& out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(g_addrs_lock);
    SymbolAddrs& a = g_addrs[dev];
    if (!a.ready) {
        void* pt = nullptr;
        void* pf = nullptr;
        if ((e = cudaGetSymbolAddress(&pt, g_noalloc_traces)) != cudaSuccess) return e;
        if ((e = cudaGetSymbolAddress(&pf, g_noalloc_flags)) != cudaSuccess) return e;
        a.traces = static_cast<double*>(pt);
        a.flags = static_cast<DevFlags*>(pf);
        a.ready = true;
    }
    out = a;
    return cudaSuccess;
}

}  // namespace

extern "C" kbl_status kbl_bounds_noalloc(const kbl_config* cfg, int n_elem, const int32_t* nbr_dev,
                                         int n_bc, const double* bc_dev, const double* w_dev,
                                         double* bnd_dev, void* cuda_stream)
{
    // the configurations kbl_create accepts, with the trapezoidal rule only
    if (!kbl_config_valid(cfg) || cfg->quadrature != 0 || n_elem < 0 || n_bc < 0) return KBL_EINVAL;
    const int n = cfg->p + 1;
    const int nv = cfg->dim + 2;
    const int ns = cfg->dim == 1 ? n : n * n;
    const int nfp = cfg->dim == 1 ? 2 : 4 * n;
    if ((unsigned long long)n_elem * nv * nfp > KBL_NOALLOC_MAX_TRACE_VALUES) return KBL_EINVAL;
    if (n_elem == 0) return KBL_OK;
    if (!nbr_dev || !w_dev || !bnd_dev || (n_bc > 0 && !bc_dev)) return KBL_EINVAL;
    SymbolAddrs a;
    cudaError_t e = symbol_addrs(a);
    if (e != cudaSuccess) return KBL_ECUDA;

    // A context on the stack that points at the caller's arrays and the static
    // scratch; it owns nothing and is never passed to kbl_destroy.
    kbl_ctx c;
    c.cfg = *cfg;
    c.phys.gamma = cfg->gamma;
    c.phys.k = cfg->k;
    c.phys.r_fac = cfg->r_fac;
    c.phys.eps = cfg->eps;
    c.phys.rho_floor = cfg->rho_floor;
    c.phys.p_floor = cfg->p_floor;
    c.phys.eps_rule = cfg->eps_rule;
    c.phys.uncoupled = cfg->uncoupled;
    c.phys.flux = cfg->flux;
    c.phys.qw = nullptr;   // trapezoidal rule: a weight table would need an allocation
    c.phys.qwf = nullptr;
    c.phys.nu[0] = cfg->nu[0];
    c.phys.nu[1] = cfg->dim == 2 ? cfg->nu[1] : 1;
    kbl_phys_derive(c.phys);
    kbl_build_fr_ops(cfg->p, c.ops);
    c.stream = (cudaStream_t)cuda_stream;
    c.nv = nv;
    c.ns = ns;
    c.nfp = nfp;
    c.nsten = ns + 2 * nfp;
    c.E = n_elem;
    c.n_bc = n_bc;
    c.mesh_ready = true;
    c.d_nbr = const_cast<int*>(reinterpret_cast<const int*>(nbr_dev));
    c.d_bc = const_cast<double*>(bc_dev);
    c.d_flags = a.flags;

    // the traces are fully rewritten before they are read; the flag word must
    // start at zero on every call (the kernels set it; this call reports non-physical
    // stencils through NaN bounds only, so the word is write-only scratch here)
    if ((e = cudaMemsetAsync(a.flags, 0, sizeof(DevFlags), c.stream)) != cudaSuccess) return KBL_ECUDA;
    if (launch_traces(&c, w_dev, a.traces, c.stream) < 0) return KBL_EINVAL;
    if (launch_bounds(&c, w_dev, a.traces, bnd_dev, c.stream) < 0) return KBL_EINVAL;
    e = cudaGetLastError();
    return e == cudaSuccess ? KBL_OK : KBL_ECUDA;
}
