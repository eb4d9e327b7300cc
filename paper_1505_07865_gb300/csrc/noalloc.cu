// ibr_op_vcycle_noalloc: the scalar multigrid V-cycles of ibr_op_vcycle for
// callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is unavailable or forbidden --
// an application that has handed all device memory to its own pool allocator,
// a plug-in loaded into a host program that owns the CUDA context, or work that
// must not block on the allocator's device-wide synchronisation.  Such callers
// provide only the right-hand side and the solution; the coarse-level buffers
// of the multigrid hierarchy come from one file-scope device array instead of
// the grid's allocations.
//
// The array is fixed at IBR_NOALLOC_SCRATCH_DOUBLES doubles (4 MiB), is held
// by every GPU that loads the library until the process exits, and is shared
// by all calls: it keeps whatever the last call left in it, and calls whose
// execution overlaps on the GPU (different streams, or different host threads)
// race on it.  No value in it needs to start at zero: every coarse-level entry
// is written before it is read.
#include <cmath>
#include <mutex>

#include "ibr_internal.cuh"

namespace ibr {
namespace {

constexpr long long IBR_NOALLOC_SCRATCH_DOUBLES = 524288;  // 4 MiB
static __device__ __align__(256) double g_noalloc_scratch[IBR_NOALLOC_SCRATCH_DOUBLES];

constexpr int kMaxDevices = 64;
static double* g_scratch_dev[kMaxDevices] = {nullptr};
static std::mutex g_scratch_mu;

// Device address of the scratch array on the current device.  The array's
// name is only a host-side stand-in in host code, so the address is looked up
// once per device (with that device current) and cached.
double* scratch_address() {
    int dev = 0;
    IBR_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) throw Error{IBR_EINVAL, "device index out of range"};
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            throw Error{IBR_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e)};
        g_scratch_dev[dev] = static_cast<double*>(p);
    }
    return g_scratch_dev[dev];
}

// same coarsening rule as the grid's hierarchy: halve while every axis is a
// multiple of 4 and the level has more than 64 cells
bool coarsenable(const Geo& g) {
    int ns[3] = {g.n0, g.n1, g.n2};
    for (int a = 0; a < g.d; ++a)
        if (ns[a] % 4 != 0) return false;
    return g.ncell > 64;
}

}  // namespace
}  // namespace ibr

using namespace ibr;

extern "C" int ibr_op_vcycle_noalloc(int dim, const int* n, const double* L, double sigma, double kappa,
                                     const double* f, double* u, int k, int pre, int post, void* cuda_stream) {
    try {
        if (dim != 2 && dim != 3) throw Error{IBR_EINVAL, "dim must be 2 or 3"};
        if (!n || !L || !f || !u) throw Error{IBR_EINVAL, "n, L, f, u must be non-NULL"};
        if (k < 1 || sigma < 0 || !(kappa > 0)) throw Error{IBR_EINVAL, "k >= 1, sigma >= 0, kappa > 0 required"};
        if (pre < 0 || post < 0 || pre + post < 1) throw Error{IBR_EINVAL, "bad smoothing sweeps"};
        for (int a = 0; a < dim; ++a)
            if (n[a] < 4 || n[a] % 2 != 0 || !(L[a] > 0)) throw Error{IBR_EINVAL, "each n[a] even >= 4, L[a] > 0"};
        double h = L[0] / n[0];
        long long cells = 1;
        for (int a = 0; a < dim; ++a) {
            if (std::fabs(L[a] / n[a] - h) > 1e-12 * h) throw Error{IBR_EINVAL, "cells must be cubes (L[a]/n[a] equal)"};
            cells *= n[a];
        }
        if (cells >= (1LL << 31)) throw Error{IBR_EINVAL, "a field must have fewer than 2^31 cells"};
        Geo lev[32];
        int nl = 0;
        lev[nl++] = make_geo(dim, n, h);
        long long need = 0;
        while (coarsenable(lev[nl - 1]) && nl < 32) {
            Geo c = lev[nl - 1];
            c.n0 /= 2;
            c.n1 /= 2;
            if (dim == 3) c.n2 /= 2;
            c.ncell = (long long)c.n0 * c.n1 * c.n2;
            c.h *= 2.0;
            lev[nl++] = c;
            need += 2 * c.ncell;  // u and f of this level
        }
        if (lev[nl - 1].ncell > 2048) throw Error{IBR_EINVAL, "grid does not coarsen to <= 2048 cells"};
        if (need > IBR_NOALLOC_SCRATCH_DOUBLES)
            throw Error{IBR_EINVAL, "coarse levels need " + std::to_string(need) + " doubles, more than the " +
                                        std::to_string(IBR_NOALLOC_SCRATCH_DOUBLES) +
                                        "-double (4 MiB) static scratch; use ibr_op_vcycle"};
        cudaStream_t s = (cudaStream_t)cuda_stream;
        double* base = scratch_address();
        double* U[32];
        double* Fw[32];
        U[0] = u;
        Fw[0] = nullptr;
        long long off = 0;
        for (int l = 1; l < nl; ++l) {
            U[l] = base + off;
            off += lev[l].ncell;
            Fw[l] = base + off;
            off += lev[l].ncell;
        }
        int coarse_sweeps = mg_coarse_sweeps(lev[nl - 1]);
        for (int it = 0; it < k; ++it)
            mg_vcycle<double>(lev, nl, U, Fw, f, 1, 0, sigma, kappa, false, pre, post, coarse_sweeps, s);
        set_error("");
        return IBR_OK;
    } catch (const Error& e) {
        set_error(std::string("ibr_op_vcycle_noalloc: ") + e.msg);
        return e.code;
    }
}
