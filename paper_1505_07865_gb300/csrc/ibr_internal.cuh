// Internal declarations shared by the translation units of libibrigid.
// Device kernels are launched only through the host wrappers declared here.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <mutex>
#include <string>
#include <utility>

#include "../../include/ibrigid.h"

namespace ibr {

// ---------------------------------------------------------------------------
// 4-point Peskin kernel: the continuous function on [-2,2] fixed by
// sum_j phi(r-j) = 1, sum_j (r-j) phi(r-j) = 0, even/odd sums 1/2 and
// sum_j phi(r-j)^2 = 3/8.
__host__ __device__ __forceinline__ double peskin4(double r) {
    r = fabs(r);
    if (r < 1.0) return 0.125 * (3.0 - 2.0 * r + sqrt(1.0 + 4.0 * r - 4.0 * r * r));
    if (r < 2.0) return 0.125 * (5.0 - 2.0 * r - sqrt(-7.0 + 12.0 * r - 4.0 * r * r));
    return 0.0;
}

// Six-point kernel of Bao, Kaye and Peskin (the kernel Sec. III.A uses):
// support [-3, 3], zeroth to third moments 1, 0, K, 0 with
// K = 59/60 - sqrt(29)/20, even and odd nodes half each, sum of squares C
// fixed at the integers.  For r in [0, 1) the weights w[m] = phi(r - (m - 2)),
// m = 0..5, follow by elimination from the five linear conditions in terms of
// t = phi(r - 3); the sum of squares leaves 28 t^2 + b t + c = C, whose root
// with t = 0 at r = 0 is taken (its discriminant stays >= 1.39 on [0, 1), so
// the branch is continuous); the root is formed without cancellation on both
// signs of b.  FP64 (set-up only).
__host__ __device__ __forceinline__ void bkp6_weights(double r, double* w) {
    const double K = 59.0 / 60.0 - sqrt(29.0) / 20.0;
    const double C = (0.625 - 0.25 * K) * (0.625 - 0.25 * K) + 0.125 + 2.0 * (0.125 * K - 0.0625) * (0.125 * K - 0.0625);
    const double r2 = r * r, r3 = r2 * r, r4 = r2 * r2, r6 = r3 * r3;
    const double b = -(84.0 * K * r + 18.0 * K + 28.0 * r3 + 18.0 * r2 - 88.0 * r - 27.0) / 12.0;
    const double c = (720.0 * K * K * r2 + 108.0 * K * K + 480.0 * K * r4 - 1416.0 * K * r2 - 396.0 * K + 80.0 * r6 -
                      436.0 * r4 + 644.0 * r2 + 603.0) /
                     1152.0;
    const double sd = sqrt(fmax(b * b - 112.0 * (c - C), 0.0));
    const double t = b >= 0.0 ? 2.0 * (C - c) / (b + sd) : (sd - b) / 56.0;
    w[0] = -0.0625 + 0.125 * K - 0.25 * K * r + r / 12.0 + 0.125 * r2 - r3 / 12.0 + t;
    w[1] = 0.25 - 2.0 * r / 3.0 + 0.5 * K * r + r3 / 6.0 - 3.0 * t;
    w[2] = 0.625 - 0.25 * K - 0.25 * r2 + 2.0 * t;
    w[3] = 0.25 + 2.0 * r / 3.0 - 0.5 * K * r - r3 / 6.0 + 2.0 * t;
    w[4] = -0.0625 + 0.125 * K + 0.25 * K * r - r / 12.0 + 0.125 * r2 + r3 / 12.0 - 3.0 * t;
    w[5] = t;
}

// The kw (4 or 6) nodes j0 .. j0 + kw - 1 of the kernel window of position s
// (grid units from node 0) and their weights phi(s - j).
__host__ __device__ __forceinline__ void kernel_window(int kw, double s, int& j0, double* w) {
    const double fl = floor(s);
    if (kw == 6) {
        j0 = (int)fl - 2;
        bkp6_weights(s - fl, w);
    } else {
        j0 = (int)fl - 1;
        for (int m = 0; m < 4; ++m) w[m] = peskin4(s - (fl - 1.0 + m));
    }
}

// ---------------------------------------------------------------------------
// errors
void set_error(const std::string& msg);
struct Error {
    int code;
    std::string msg;
};
#define IBR_CUDA_TRY(expr)                                                         \
    do {                                                                          \
        cudaError_t _e = (expr);                                                  \
        if (_e != cudaSuccess)                                                    \
            throw ::ibr::Error{IBR_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)}; \
    } while (0)
// every kernel launch of the library goes through this check (and counter);
// add_launches accounts for the kernels of a replayed CUDA graph
void count_launch();
void add_launches(long long n);
long long thread_launches();  // launches counted on the calling thread
bool profiling_enabled();
#define IBR_CHECK_LAUNCH()                  \
    do {                                    \
        ::ibr::count_launch();              \
        IBR_CUDA_TRY(cudaGetLastError());   \
    } while (0)

// Programmatic dependent launch for chains of dependent kernels on one
// stream (the V-cycle, P_S): a kernel launched by launch_k may be scheduled
// while its predecessor drains (its launch latency overlaps the predecessor's
// last wave); it lets its own successor do the same (pdl_start) and waits for
// the predecessor's results in hardware (griddepcontrol.wait) before reading
// any input.  Kernels launched this way call pdl_start() first; outside a
// programmatic launch both are no-ops.  IBR_PDL=0 in the environment: plain
// launches.
__device__ __forceinline__ void pdl_start() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
bool pdl_enabled();

// Bulk asynchronous copies into shared memory with completion counted on an
// mbarrier (the producer / consumer pipelines of the tensor-core products and
// of the double-float Gram-Schmidt passes).  Every wait is bounded: after
// MBAR_WAIT_LIMIT_NS the caller gets false, records an error and stops.
constexpr unsigned long long MBAR_WAIT_LIMIT_NS = 4000000000ULL;  // 4 s per wait
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    const unsigned long long t0 = global_ns();
    for (long long it = 0;; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 255) == 255 && global_ns() - t0 > MBAR_WAIT_LIMIT_NS) return false;
    }
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}
template <typename... KArgs, typename... Args>
void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    IBR_CUDA_TRY(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
}

// Runs a set-up step (e.g. cudaFuncSetAttribute, which acts on the current
// device only) once per CUDA device, from any host thread: the step runs with
// the device current, under a lock, the first time run() is called on it.
class PerDeviceOnce {
  public:
    template <typename F>
    void run(F&& fn) {
        int dev = 0;
        IBR_CUDA_TRY(cudaGetDevice(&dev));
        if (dev < 0 || dev >= 128) throw Error{IBR_EINVAL, "device index out of range"};
        std::lock_guard<std::mutex> lk(mu_);
        const unsigned long long bit = 1ULL << (dev & 63);
        if (done_[dev >> 6] & bit) return;
        fn();
        done_[dev >> 6] |= bit;
    }

  private:
    std::mutex mu_;
    unsigned long long done_[2] = {0ULL, 0ULL};
};

// kernel classes timed by the optional profiler (prof.cu)
enum KernelId {
    KID_STOKES, KID_RBGS, KID_RESTRICT, KID_PROLONG, KID_COARSE, KID_PS_DIV, KID_PS_FINISH,
    KID_AXPBY, KID_SCALE, KID_CONVERT, KID_MDOT, KID_UPD_MDOT, KID_UPD_NORM, KID_NORM2, KID_COMBINE,
    KID_BLOCK_MEANS, KID_SUB_MEANS, KID_SMALL, KID_SPREAD, KID_INTERP, KID_LAMSUM, KID_RIGID_K,
    KID_RIGID_KT, KID_MARKERS, KID_MTILDE, KID_SPD_INV, KID_GEMV, KID_ADVECT, KID_TC_GEMM, KID_COUNT
};
// records CUDA events around the launches in its scope when profiling is on;
// bytes = the algorithmic bytes those launches move, flops = the
// floating-point operations they execute (tensor-core products; 0 elsewhere)
// One timed region of the CUDA-event profile: count back-to-back launches of
// one kernel class between two events (bytes and flops are their totals), so
// that a sequence of short dependent launches is timed as it runs, without an
// event between each pair.
class ProfScope {
  public:
    ProfScope(int kid, cudaStream_t s, double bytes, double flops = 0.0, int count = 1);
    ~ProfScope();
    ProfScope(const ProfScope&) = delete;
    ProfScope& operator=(const ProfScope&) = delete;

  private:
    int kid_;
    cudaStream_t s_;
    double bytes_, flops_;
    int count_;
    void* a_;
};

// ---------------------------------------------------------------------------
// cell grid (x fastest); n2 == 1 in 2-D.  wall: bit a set when axis a is
// bounded by walls at both ends (else periodic).  Along a wall axis the
// cell-centred fields and the tangential velocity components hold the n cell
// centres; the normal component holds faces 0..n-1, face 0 on the low wall (a
// boundary entry whose equation is `value = wall data`), face n (high wall)
// not stored.
struct Geo {
    int d;
    int n0, n1, n2;
    long long ncell;
    double h;
    int wall;
    int kw;  // support of the kernel of J and S: 4 (Peskin) or 6 (Bao, Kaye, Peskin)
};

// field codes of the stencil and multigrid kernels: velocity components
// 0..d-1, the pressure (cell-centred, homogeneous Neumann on walls) FLD_P
constexpr int FLD_P = 3;

inline Geo make_geo(int d, const int* n, double h) {
    Geo g;
    g.d = d;
    g.n0 = n[0];
    g.n1 = n[1];
    g.n2 = d == 3 ? n[2] : 1;
    g.ncell = (long long)g.n0 * g.n1 * g.n2;
    g.h = h;
    g.wall = 0;
    g.kw = 4;
    return g;
}

inline int grid_1d(long long work, int block) {
    long long b = (work + block - 1) / block;
    if (b < 1) b = 1;
    if (b > 2147483647LL) b = 2147483647LL;
    return (int)b;
}

// ---------------------------------------------------------------------------
// stencil.cu -- MAC operators and multigrid (templated on scalar T)
// y = [A v + G p + shift ; -D v] for the unconstrained Stokes operator
// (walls: homogeneous boundary conditions; wall-face rows are the identity).
template <typename T>
void stokes_apply(const Geo& g, const T* x, T* y, double sigma, double eta, const double* shift_dev,
                  cudaStream_t s);
// The multigrid pieces act on C stacked fields with field codes fld0,
// fld0 + 1, ... (fld0 == FLD_P: one pressure field), which fix the boundary
// rule of each field on wall axes.
// red-black Gauss-Seidel half sweep: (sigma u - kappa Delta_h u) = f
template <typename T>
void mg_smooth(const Geo& g, T* u, const T* f, int C, int fld0, double sigma, double kappa, int color,
               bool zero_init, cudaStream_t s);
template <typename T>
void mg_residual_restrict(const Geo& gf, const Geo& gc, const T* u, const T* f, T* fc, int C, int fld0,
                          double sigma, double kappa, cudaStream_t s);
template <typename T>
void mg_prolong_correct(const Geo& gf, const Geo& gc, T* u, const T* uc, int C, int fld0, cudaStream_t s);
template <typename T>
void mg_coarse_solve(const Geo& g, T* u, const T* f, int C, int fld0, double sigma, double kappa, int sweeps,
                     cudaStream_t s);
// One V-cycle for (sigma I - kappa Delta_h) U[0] = F0 on the levels lev[0..L)
// (C stacked fields): red-black pre/post sweeps, averaging restriction into
// Fw[l] (l >= 1), (bi/tri)linear prolongation, coarsest level by red-black
// sweeps in one CTA; all levels with <= MG_TAIL_MAX_CELLS cells run inside one
// shared-memory kernel.  zero_start: U[0] starts at zero (else from its value).
constexpr int MG_TAIL_MAX_LEVELS = 8;
constexpr long long MG_TAIL_MAX_CELLS = 4096;
constexpr size_t MG_TAIL_MAX_SMEM = 200 * 1024;
// rb_u, rb_f: scratch of C * lev[0].ncell each (or NULL): with them a periodic
// 3-D finest level (n0 a multiple of 8) of a zero-start V-cycle with pre, post
// >= 1 runs in red-black split layout (the same arithmetic, bitwise); rb_u1,
// rb_f1 (C * lev[1].ncell each, or NULL) do the same for level 1
template <typename T>
void mg_vcycle(const Geo* lev, int L, T* const* U, T* const* Fw, const T* F0, int C, int fld0, double sigma,
               double kappa, bool zero_start, int pre, int post, int coarse_sweeps, cudaStream_t s,
               T* rb_u = nullptr, T* rb_f = nullptr, T* rb_u1 = nullptr, T* rb_f1 = nullptr);
// red-black sweeps of the coarsest-level solve: enough for a preconditioner
// (the coarsest grid has at most a few hundred cells)
inline int mg_coarse_sweeps(const Geo& g) {
    int nmax = g.n0 > g.n1 ? g.n0 : g.n1;
    if (g.n2 > nmax) nmax = g.n2;
    return 2 * nmax > 8 ? 2 * nmax : 8;
}
// raises the shared-memory limit of the tail kernel (call outside stream capture)
template <typename T>
void mg_set_attributes();
// times the half-sweep tiles of a periodic 3-D level (C stacked fields) once
// per level shape and keeps the fastest (no-op elsewhere and during capture)
template <typename T>
void mg_tune_smoother(const Geo& g, int C, cudaStream_t s);
// tuned tile idx: n0, n1, n2, C, element size, by, kz (false past the end)
bool tuned_tile(int idx, int* out7);
// times the V-cycle schedules of a periodic 3-D hierarchy (per-level kernels,
// or the thread-block-cluster kernel from each feasible level) once per
// hierarchy shape and keeps the fastest (no-op elsewhere and during capture);
// U[1..L), Fw[1..L): the hierarchy's level buffers, used as scratch
template <typename T>
void mg_tune_cluster(const Geo* lev, int L, T* const* U, T* const* Fw, int C, int coarse_sweeps, cudaStream_t s);
// tuned schedule idx: n0, n1, n2, levels, C, element size, first cluster
// level (-2: none) (false past the end)
bool tuned_cluster(int idx, int* out7);
// q = -D y - hd ; (P_S middle factor, Sec. V.B)
template <typename T>
void ps_divergence(const Geo& g, const T* y, const T* hd, T* q_rhs, double rhs_scale, T* q, cudaStream_t s);
// v = y + h^2 G phi ; pi = c_q q + c_phi phi   (P_S first factor)
template <typename T>
void ps_finish(const Geo& g, const T* y, const T* phi, const T* q, T* z, double c_q, double c_phi,
               cudaStream_t s);
// Boundary data of wall `side` (0 low, 1 high) of wall axis a moved into the
// right-hand side b = [g_0 .. g_{d-1} | h] (FP64): wall-face rows of the
// normal component set to the wall value, data terms of the neighbouring
// rows added (App. D extension with data).  data: [d][face points], the
// face points ordered over the other axes, lower axis fastest.
void wall_lift(const Geo& g, int a, int side, const double* data, double* b, double eta, cudaStream_t s);
// x's stored low-wall faces of component a set to the wall value (their rows
// are the identity and nothing else couples to them)
void wall_set_faces(const Geo& g, int a, const double* data, double* x, cudaStream_t s);

// ---------------------------------------------------------------------------
// advect.cu -- explicit advection of the time-stepped problems (FP64)
// wall velocities per wall side 2a + s ([d][face points]; NULL on periodic axes)
struct WallData {
    const double* data[6];
};
// N = div(v v), centred flux form, App. D extension with the wall data
void advect(const Geo& g, const double* v, const WallData& wd, double* N, cudaStream_t s);
// out = sigma v - (rho_c1 Nn + rho_c0 Np) + f   (f may be NULL), m entries
void step_force(long long m, const double* v, const double* Nn, const double* Np, const double* f, double sigma,
                double rho_c1, double rho_c0, double* out, cudaStream_t s);

// ---------------------------------------------------------------------------
// blas.cu -- vector kernels; dots reduce deterministically (fixed blocks)
constexpr int RED_BLOCKS = 608;   // 4 x 152 SMs
constexpr int RED_THREADS = 256;
constexpr int MDOT_CHUNK = 8;
template <typename T>
void vec_axpby(long long n, double a, const T* x, double b, T* y, cudaStream_t s);   // y = a x + b y
template <typename T>
void vec_scale_copy(long long n, const double* scale_dev, bool invert, const T* x, T* y,
                    cudaStream_t s);  // y = x * (invert ? 1/scale : scale)
template <typename Ti, typename To>
void vec_convert(long long n, const Ti* x, To* y, cudaStream_t s);
// partial dots of w against k vectors V + j*ld, summed into out[0..k) (double)
template <typename T>
void mdot(long long n, const T* V, long long ld, int k, const T* w, double* partial, double* out,
          cudaStream_t s);
// w -= sum_j h[j] V_j, then out[j] = V_j . w (CGS2 second pass); h device
template <typename T>
void update_mdot(long long n, const T* V, long long ld, int k, const double* h, T* w, double* partial,
                 double* out, cudaStream_t s);
// w -= sum_j h[j] V_j, then out[0] = w . w
template <typename T>
void update_norm2(long long n, const T* V, long long ld, int k, const double* h, T* w, double* partial,
                  double* out, cudaStream_t s);
template <typename T>
void norm2(long long n, const T* w, double* partial, double* out, cudaStream_t s);
// x (+)= sum_j y[j] Z_j  (y device)
template <typename T, typename Tz>
void combine(long long n, const Tz* Z, long long ld, int k, const double* y, T* x, bool accumulate,
             cudaStream_t s);
// means of C consecutive blocks of length m (partial sums, double), then
// x_c -= mean_c for the blocks selected by mask
template <typename T>
void block_means(long long m, int C, const T* x, double* partial, double* out, cudaStream_t s);
template <typename T>
void subtract_means(long long m, int C, T* x, const double* means, cudaStream_t s);

// One Arnoldi step's orthonormalisation against V_0..V_{k-1} (classical
// Gram-Schmidt, second pass only when |w_perp|^2 < |w|^2 / 2):
//   h1[0..k) = V^T w, h1[k] = |w|^2; h2 = second-pass coefficients (or 0);
//   st[2] = |w_perp|^2; vout = w_perp / |w_perp| (vout may alias w);
//   out2[0..n2) = vout[0..n2) converted to T2 (if out2 != NULL).
// h1, hk2 hold k+1 doubles; h2 k; st 3; partial RED_BLOCKS*(k+1).
template <typename T, typename T2>
void cgs_orthonormalize(long long n, const T* V, long long ld, int k, T* w, T* vout, T2* out2, long long n2,
                        double* partial, double* h1, double* h2, double* hk2, double* st, cudaStream_t s);
// Only the Hessenberg column of the last step of a GMRES cycle whose next
// basis vector is never used: h1 = V^T w (one pass), h2 = 0, st[2] =
// max(|w|^2 - |h1|^2, 0) (no second pass, no normalisation pass)
template <typename T>
void cgs_coeffs_only(long long n, const T* V, long long ld, int k, const T* w, double* partial, double* h1,
                     double* h2, double* st, cudaStream_t s);
// y = x * (*inv_norm) (the 1/|x| formed by givens_init), plus optional out2[0..n2) copy
template <typename T, typename T2>
void scale_rsqrt(long long n, const double* inv_norm, const T* x, T* y, T2* out2, long long n2, cudaStream_t s);

// The outer FGMRES basis in double-float: value = hi + lo (48-bit
// significand), 8 bytes per entry like FP64; its Gram-Schmidt passes run on
// the FP32 pipe (error-free two-sum / two-product).
struct __align__(8) dflt {
    float hi, lo;
};
// Modified Gram-Schmidt of w against the FP64 basis V_0..V_{k-1} (rows of
// ld doubles) and V_k = the normalised remainder into vout, with an FP32 copy
// of its first n32 entries (out32, may be NULL): h[0..k) the coefficients,
// st[2] = |w_perp|^2, st[3] its inverse square root, st[1] = 0.  k + 2
// launches, two FP64 FMAs per entry and basis vector; w is overwritten.  n and
// ld even (entries past the system length are a zero pad of w and of every
// basis vector), V, w, vout 16-byte aligned; partial holds 2 * 760 doubles.
void mgs_orthonormalize(long long n, const double* V, long long ld, int k, double* w, double* vout, float* out32,
                        long long n32, double* partial, double* h, double* st, cudaStream_t s);
// cgs_orthonormalize of the outer FGMRES basis, pipelined on bulk copies: V
// is FP64 or (df) double-float, 8 bytes per entry either way; w is FP64 on
// entry (double-float: converted in place, w's contents are consumed); the
// same passes and outputs (h1, h2, hk2, st); vout = the new basis vector;
// out32 (first n32 entries, float) and out64 (entries from64..n_real-1, FP64)
// copies of it for the preconditioner (either may be NULL).  n and ld even
// (entries n_real..n-1 are a zero pad of w and of every basis vector), V, w
// and vout 16-byte aligned, 1 <= k <= 128; partial holds 304 * (k + 1)
// doubles.  A wait that times out sets *err (device int).
void cgs_orthonormalize_pipe(bool df, long long n, long long n_real, const void* V, long long ld, int k, double* w,
                             void* vout, float* out32, long long n32, double* out64, long long from64,
                             double* partial, double* h1, double* h2, double* hk2, double* st, int* err,
                             cudaStream_t s);
// vout = x * (*inv_norm) in double-float (n entries), with the same copies
void scale_df(long long n, long long n_real, const double* inv_norm, const double* x, dflt* vout, float* out32,
              long long n32, double* out64, long long from64, cudaStream_t s);

// small single-thread kernels for the Arnoldi/Givens bookkeeping (FP64)
// H column j (k = j+2 entries) assembled from h1 + h2 and the norm; Givens
// rotations applied, new rotation formed, res_out = |g[j+1]|.
void arnoldi_column(double* H, int ldh, const double* h1, const double* h2, const double* nrm2, int j,
                    double* cs, double* sn, double* gv, double* res_out, double* inv_norm_out,
                    cudaStream_t s);
// g = [beta, 0, ...]; beta from nrm2 (sqrt), inv_beta out
void givens_init(const double* nrm2, double* gv, int m1, double* beta_out, double* inv_beta_out,
                 cudaStream_t s);
void hess_solve(const double* H, int ldh, const double* gv, int k, double* y, cudaStream_t s);

// ---------------------------------------------------------------------------
// ib.cu -- markers, kernel weights, spread gather lists, J, S, K, K^T
struct MarkerData {
    int N = 0;
    int B = 0;
    double* q = nullptr;        // [N][d] lab positions (wrapped)
    double* rel = nullptr;      // [N][d] q - X_body (unwrapped lever arm)
    int* body = nullptr;        // [N]
    int* body_start = nullptr;  // [B+1]
    int* idx = nullptr;         // [N][d][d][kw] stored node of window node m, comp alpha, axis beta
    double* w64 = nullptr;      // [N][d][d][kw] signed weights (mirror images carry -1)
    float* w32 = nullptr;       // [N][d][d][kw]
    // face-major gather lists of S: faces F, entries E
    long long F = 0, E = 0;
    long long* face = nullptr;  // [F] alpha*ncell + cell
    int* off = nullptr;         // [F+1]
    int* ent_m = nullptr;       // [E] marker*d + alpha
    double* ent_w64 = nullptr;  // [E]
    float* ent_w32 = nullptr;   // [E]
};
void markers_positions(int d, int N, const double* rbody, const int* body, const double* xc_R /*[B][12]*/,
                       const double* Lbox, double* q, double* rel, cudaStream_t s);
void markers_weights(const Geo& g, int N, const double* q, int* idx, double* w64, float* w32,
                     cudaStream_t s);
// builds the face-major gather lists (allocates md.face/off/ent_* on device)
void markers_build_gather(const Geo& g, MarkerData& md, cudaStream_t s);
// y[face] += scale * sum w * lam   (no atomics; one thread per touched face)
template <typename T>
void spread_gather(const MarkerData& md, const T* lam, T* y, double scale, cudaStream_t s);
// out[i*d+a] = sign * (J v)_i^a + (add ? add_scale * add[i*d+a] : 0)
template <typename T, typename Tadd>
void interp(const Geo& g, const MarkerData& md, const T* v, T* out, double sign, const Tadd* add,
            cudaStream_t s, double add_scale);
// shift[a] = scale * sum_i lam[i*d+a]  (double, a < d)
template <typename T>
void lam_sum(int d, int N, const T* lam, double scale, double* shift, cudaStream_t s);
void rigid_K(int d, int N, const double* rel, const int* body, const double* UO, double* V, double sign,
             cudaStream_t s);
void rigid_KT(int d, int B, const int* body_start, const double* rel, const double* lam, double* FT,
              cudaStream_t s);

// free kinematics: bfree[b] = index of body b among the free bodies or -1;
// U_f and the per-body outputs are body-major with nr = d + rot entries.
void rigid_K_free(int d, int N, const double* rel, const int* body, const int* bfree, const double* Uf, double* out,
                  double sign, cudaStream_t s);  // out += sign K_f U_f
template <typename Tl>
void rigid_KT_free(int d, int B, const int* bstart, const int* bfree, const double* rel, const Tl* lam, double* out,
                   cudaStream_t s);  // out = K_f^T lam
template <typename T>
void lam_add_XU(int d, int N, const int* body, const int* bfree, const T* X, const double* Uf, T* lam,
                cudaStream_t s);  // lam += X U_f, X = nr columns of length dN
void body_solve(int nfree, int nr, const double* Nb, const double* r, const double* sv, double* U,
                cudaStream_t s);  // U = Nb (r - sv)
void small_inverse(int nfree, int nr, double* A, int* info, cudaStream_t s);

// ---------------------------------------------------------------------------
// dense.cu -- approximate mobility blocks
struct MobParams {
    int model;        // IBR_MOB_RPY or IBR_MOB_FIT2D
    double eta, h, l, a;
    double corr;      // periodic correction subtracted from f (3-D)
    double coef[9];
    double box[3];    // periodic box lengths (0 on wall axes): displacements are minimum images
};
void mtilde_build(int d, int Nb, const double* rel_b, const MobParams& p, double* M, cudaStream_t s);
// in place: M (n x n, row-major, SPD) -> M^-1 (full symmetric).  info_dev[0]
// set to (k+1) if the k-th pivot is <= min_pivot.  work >= n*n.
// The pair-mobility table of a periodic grid: for S source points x0[s]
// and force directions beta, the velocity field v = L^-1 S~ (unit force
// e_beta at x0[s]) stored in FP32 as tab[((s*d + beta)*d + alpha)*ncell + cell]
// (alpha: velocity component).  pair_mtilde builds the dense block of the
// nr markers at positions q[nr][d] (row-major, (d nr)^2):
//   M~_ij^{ab} = (1/2S) sum_s [ J_a(x0_s + q_i - q_j) v^{s,b} + J_b(x0_s + q_j - q_i) v^{s,a} ]
// (exactly symmetric).  point_spread writes y[beta*ncell + .] = scale * the
// 4^d kernel weights of component beta at x0 (periodic; other entries untouched).
void pair_mtilde(const Geo& g, int nr, const double* q, int S, const double* x0, const float* tab, double* M,
                 cudaStream_t s);
void point_spread(const Geo& g, const double* x0, int beta, double scale, double* y, cudaStream_t s);
template <typename T>
void spd_inverse(int n, T* M, T* work, int* info_dev, double min_pivot, cudaStream_t s);
template <typename Ti, typename To>
void mat_convert(long long n, const Ti* a, To* b, cudaStream_t s);
// tc_gemm.cu -- tensor-core (tcgen05, split TF32) dense products:
// C = beta C + alpha A B^T, A [M][K], B [N][K] row-major FP32; M, N multiples
// of 128, K of 32; lower_only: the 128 x 128 tiles above the diagonal are
// not computed; err_dev[0] = 1 if a wait for the tensor cores timed out
void gemm_tf32x3(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc, float alpha,
                 float beta, bool lower_only, int* err_dev, cudaStream_t s);
// M (n x n SPD FP32) -> M^-1 with the tensor-core products (blocked Cholesky,
// triangular inverse, X^T X); info_dev as in spd_inverse; pad: the diagonal
// of the identity block that pads n to a multiple of 128
void spd_inverse_tc(int n, float* M, int* info_dev, double min_pivot, double pad, int* err_dev, cudaStream_t s);
template <typename T>
void add_diag(int n, T* M, double delta, cudaStream_t s);   // M += delta I
// out[r] = sum_c Minv_b[r][c] rhs[c] for each body block (offsets in elements)
template <typename T, typename Tv>
void blockdiag_gemv(int B, const long long* moff_dev, const int* roff_dev, int max_rows, const T* Mall,
                    const Tv* rhs, Tv* out, cudaStream_t s);

}  // namespace ibr
