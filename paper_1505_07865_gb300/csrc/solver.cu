// Host orchestration and the C ABI of libibrigid.
//
// Outer solver: right-preconditioned flexible GMRES in FP64 on the
// constrained system (Sec. V), Arnoldi by classical Gram-Schmidt with a
// second pass only when needed, Givens rotations on the device, true residual
// recomputed at every restart and at exit.
// Preconditioner: the Schur-complement preconditioner of Sec. V.A
//   1. inner GMRES(N_s) on the unconstrained Stokes system, each step
//      preconditioned by P_S (Sec. V.B, Eq. P1_practical) = one vector
//      V-cycle for A~^-1, the divergence, one scalar V-cycle for L~p^-1,
//      the gradient correction and B~^-1;
//   2. dU = -(J v + W);  3. Lambda = M~^-1 dU (Eq. mob_subproblem);
//   4. (full variant) a second inner solve with g + S~ Lambda.
// The preconditioner runs in FP32 (IBR_MIXED) or FP64 (IBR_FP64).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "ibr_internal.cuh"

namespace ibr {
static thread_local std::string g_last_error;
void set_error(const std::string& m) { g_last_error = m; }
}  // namespace ibr

using namespace ibr;

namespace {

template <typename T>
T* dalloc(size_t n) {
    T* p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc(&p, n * sizeof(T));
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        throw Error{IBR_ENOMEM, std::string("cudaMalloc of ") + std::to_string(n * sizeof(T)) +
                                    " bytes failed: " + cudaGetErrorString(e)};
    }
    return p;
}
template <typename T>
void dfree(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// ---------------------------------------------------------------------------
// geometric multigrid on cell grids (C stacked fields, periodic or wall axes)
template <typename T>
struct Multigrid {
    std::vector<Geo> lev;
    std::vector<T*> u, f;  // index 0 unused (caller's buffers)
    T *rb_u = nullptr, *rb_f = nullptr;    // finest level in red-black split layout (periodic 3-D)
    T *rb_u1 = nullptr, *rb_f1 = nullptr;  // level 1 in the same layout
    int cmax = 0;
    int coarse_sweeps = 40;

    static bool can_coarsen(const Geo& g) {
        int ns[3] = {g.n0, g.n1, g.n2};
        // the coarse grid must stay even on every axis (red-black ordering)
        for (int a = 0; a < g.d; ++a)
            if (ns[a] % 4 != 0) return false;
        return g.ncell > 64;
    }
    void init(const Geo& g0, int cmax_) {
        release();
        cmax = cmax_;
        lev.push_back(g0);
        u.push_back(nullptr);
        f.push_back(nullptr);
        Geo g = g0;
        while (can_coarsen(g)) {
            Geo c = g;
            c.n0 /= 2;
            c.n1 /= 2;
            if (g.d == 3) c.n2 /= 2;
            c.ncell = (long long)c.n0 * c.n1 * c.n2;
            c.h = g.h * 2.0;
            lev.push_back(c);
            u.push_back(dalloc<T>((size_t)cmax * c.ncell));
            f.push_back(dalloc<T>((size_t)cmax * c.ncell));
            g = c;
        }
        coarse_sweeps = mg_coarse_sweeps(lev.back());
        if (g0.d == 3 && !g0.wall && g0.n0 % 8 == 0 && lev.size() > 1) {
            rb_u = dalloc<T>((size_t)cmax * g0.ncell);
            rb_f = dalloc<T>((size_t)cmax * g0.ncell);
        }
        if (g0.d == 3 && !g0.wall && lev.size() > 2 && lev[1].n0 % 8 == 0) {
            rb_u1 = dalloc<T>((size_t)cmax * lev[1].ncell);
            rb_f1 = dalloc<T>((size_t)cmax * lev[1].ncell);
        }
    }
    void release() {
        dfree(rb_u);
        dfree(rb_f);
        dfree(rb_u1);
        dfree(rb_f1);
        for (auto& p : u) dfree(p);
        for (auto& p : f) dfree(p);
        u.clear();
        f.clear();
        lev.clear();
    }
    // one V-cycle for (sigma I - kappa Delta_h) u0 = f0 (C stacked fields)
    // fld0: field code of the first stacked field (velocity component, or FLD_P)
    void vcycle(T* u0, const T* f0, int C, int fld0, double sigma, double kappa, bool zero_start, int pre, int post,
                cudaStream_t s) {
        int L = (int)lev.size();
        std::vector<T*> U(u);
        U[0] = u0;
        mg_vcycle<T>(lev.data(), L, U.data(), f.data(), f0, C, fld0, sigma, kappa, zero_start, pre, post,
                     coarse_sweeps, s, rb_u, rb_f, rb_u1, rb_f1);
    }
};

struct Body {
    double xc[3] = {0, 0, 0};
    double R[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    int kin = IBR_PRESCRIBED;
    std::vector<double> rbody;
    int N = 0;
};

}  // namespace

// IBR_MOB_PAIR: source points of the pair-mobility table, inner GMRES length
// of its solves, largest d N of one dense block for all markers
constexpr int PAIR_S = 2;
constexpr int PAIR_NS = 8;
constexpr long long PAIR_FULL_MAX_DEFAULT = 6144;
// IBR_PAIR_FULL_MAX in the environment overrides the single-block limit
long long pair_full_max() {
    static const long long v = [] {
        const char* e = std::getenv("IBR_PAIR_FULL_MAX");
        const long long x = e ? std::atoll(e) : 0;
        return x > 0 ? x : PAIR_FULL_MAX_DEFAULT;
    }();
    return v;
}

template <typename T>
struct PC;

struct ibr_grid {
    int d = 3;
    int n[3] = {1, 1, 1};
    double L[3] = {1, 1, 1};
    double h = 1, eta = 1, rho = 0, dt = 0, vol = 1;
    int precision = IBR_MIXED;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Geo geo;
    std::vector<Body> bodies;
    bool dirty = true;
    ibr_solve_opts prepared_opts;
    MarkerData md;
    int N = 0;
    long long nS = 0, len = 0;
    // free kinematics: bodies with unknown velocity under a given load
    int nfree = 0, nU = 0;   // free bodies, their unknowns ((d + rot) each)
    std::vector<int> bfree;  // body -> free index or -1
    int* bfree_dev = nullptr;
    // mobility
    std::vector<long long> moff;
    std::vector<int> roff;
    long long* moff_dev = nullptr;
    int* roff_dev = nullptr;
    int nblk = 0;              // dense mobility blocks (one per body, or one for all markers when coupled)
    double* Mbuild = nullptr;  // M~ (or M0) as built (FP64)
    double* Minv64 = nullptr;
    float* Minv32 = nullptr;
    int* info_dev = nullptr;
    std::vector<double> mob_shift;  // diagonal shift used per body (0: M~ was SPD)
    // the pair-mobility table of IBR_MOB_PAIR (periodic grids): PAIR_S source
    // points, d force directions, d velocity components, FP32; built once per grid
    float* pair_tab = nullptr;
    double* pair_x0 = nullptr;
    std::shared_ptr<void> pair_hold;  // keeps the shared table alive
    // outer FGMRES workspace
    int m_alloc = 0;
    long long len_alloc = 0;
    long long w_len = 0;  // the len w's zero pad was last set for
    // V: the basis, FP64 (or, with IBR_ARNOLDI=df, double-float: dflt, 8
    // bytes per entry); vk64: in the double-float case the FP64 copy of the
    // current basis vector that the preconditioner reads
    double *V = nullptr, *Z = nullptr, *b = nullptr, *x = nullptr, *w = nullptr, *vk64 = nullptr;
    double *H = nullptr, *cs = nullptr, *sn = nullptr, *gv = nullptr, *yv = nullptr;
    double *h1 = nullptr, *h2 = nullptr, *sc = nullptr, *partial = nullptr, *shift = nullptr, *means = nullptr;
    double *hk2 = nullptr, *st = nullptr;
    int* wait_err = nullptr;    // set by a pipelined Gram-Schmidt pass whose wait timed out
    double* host_sc = nullptr;  // pinned
    double* FT = nullptr;
    double* UO = nullptr;
    bool have_solution = false;
    PC<double>* pc64 = nullptr;
    PC<float>* pc32 = nullptr;
    int pc_ns = 0;

    bool steady() const { return rho == 0.0 || dt == 0.0; }
    double sigma() const { return steady() ? 0.0 : rho / dt; }
    // walls on some axis (geo.wall != 0), and their boundary data: bc[2a + s]
    // per side, wdata[2a + s] the velocity on that wall ([d][face points],
    // device; zero for no-slip), wdata_host the same on the host
    int bc[6] = {IBR_PERIODIC, IBR_PERIODIC, IBR_PERIODIC, IBR_PERIODIC, IBR_PERIODIC, IBR_PERIODIC};
    double* wdata[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    std::vector<double> wdata_host[6];
    bool walls() const { return geo.wall != 0; }
    // periodic steady Stokes: <v> = 0 is part of the problem and S~ = S - vol^-1 1^T
    bool null_v() const { return steady() && !walls(); }
    long long face_points(int a) const { return geo.ncell / n[a]; }
    long long len_pad() const { return (len + 1) & ~1LL; }
    // time stepping (ibr_advance): v^n, N(v^n), N(v^{n-1}), the step forcing,
    // the constant body force; hist: N(v^{n-1}) is valid (AB2 from then on)
    double *adv_v = nullptr, *adv_N = nullptr, *adv_Np = nullptr, *adv_g = nullptr, *adv_f = nullptr;
    bool adv_hist = false;
    int rot() const { return d == 2 ? 1 : 3; }
};

// ---------------------------------------------------------------------------
// preconditioner state in precision T
template <typename T>
struct PC {
    ibr_grid* G = nullptr;
    int ns = 2;
    Multigrid<T> mg;
    T *Vi = nullptr, *Zi = nullptr, *w = nullptr, *rs = nullptr, *rs2 = nullptr, *xs = nullptr;
    T *y = nullptr, *phi = nullptr, *q = nullptr, *qr = nullptr, *dU = nullptr, *lamT = nullptr;
    double *Hi = nullptr, *cs = nullptr, *sn = nullptr, *gv = nullptr, *yv = nullptr, *h1 = nullptr, *h2 = nullptr;
    double *sc = nullptr, *partial = nullptr, *means = nullptr, *shift = nullptr, *hk2 = nullptr, *st = nullptr;
    const T* Minv = nullptr;
    int pre = 2, post = 2, variant = IBR_PC_LOWER;
    long long ps_count = 0;
    // the preconditioner body (from rs and rL to xs and lamT) captured once as a
    // CUDA graph and replayed; invalidated by a new geometry or new options
    double* rL = nullptr;  // FP64 copy of the constraint part of the input
    // free bodies: X = M~^-1 K_f (nr columns of length dN), the FP64 body blocks
    // Nb = (K_f^T M~^-1 K_f)^-1, and the load / velocity vectors of the apply
    T* Xf = nullptr;
    double *Nb = nullptr, *rU = nullptr, *sU = nullptr, *Uo = nullptr;
    bool free_ready = false;
    cudaGraphExec_t gexec = nullptr;
    int g_ns = -1, g_pre = -1, g_post = -1, g_variant = -1;
    long long g_launches = 0;

    void invalidate_graph() {
        if (gexec) cudaGraphExecDestroy(gexec);
        gexec = nullptr;
    }

    PC(ibr_grid* g, int ns_) : G(g), ns(ns_) {
        long long n = G->geo.ncell;
        long long nS = G->nS;
        mg.init(G->geo, G->d);
        mg_set_attributes<T>();
        // smoother tiles of the levels (d stacked velocity components, and the pressure)
        for (const Geo& lg : mg.lev) {
            mg_tune_smoother<T>(lg, G->d, G->stream);
            mg_tune_smoother<T>(lg, 1, G->stream);
        }
        // V-cycle schedule (where the cluster kernel takes over), velocity and pressure
        for (int C : {G->d, 1})
            mg_tune_cluster<T>(mg.lev.data(), (int)mg.lev.size(), mg.u.data(), mg.f.data(), C, mg.coarse_sweeps,
                               G->stream);
        Vi = dalloc<T>((size_t)(ns + 1) * nS);
        Zi = dalloc<T>((size_t)ns * nS);
        w = dalloc<T>(nS);
        rs = dalloc<T>(nS);
        rs2 = dalloc<T>(nS);
        xs = dalloc<T>(nS);
        y = dalloc<T>((size_t)G->d * n);
        phi = dalloc<T>(n);
        q = dalloc<T>(n);
        qr = dalloc<T>(n);
        Hi = dalloc<double>((size_t)(ns + 1) * (ns + 1));
        cs = dalloc<double>(ns + 1);
        sn = dalloc<double>(ns + 1);
        gv = dalloc<double>(ns + 2);
        yv = dalloc<double>(ns + 1);
        h1 = dalloc<double>(ns + 2);
        h2 = dalloc<double>(ns + 1);
        hk2 = dalloc<double>(ns + 2);
        st = dalloc<double>(4);
        sc = dalloc<double>(8);
        partial = dalloc<double>((size_t)RED_BLOCKS * std::max(ns + 1, 4));
        means = dalloc<double>(4);
        shift = dalloc<double>(4);
        alloc_markers();
    }
    void alloc_markers() {
        invalidate_graph();
        dfree(dU);
        dfree(lamT);
        dfree(rL);
        dfree(Xf);
        dfree(Nb);
        dfree(rU);
        dfree(sU);
        dfree(Uo);
        free_ready = false;
        long long dN = (long long)G->N * G->d;
        dU = dalloc<T>(std::max(dN, 1LL));
        lamT = dalloc<T>(std::max(dN, 1LL));
        rL = dalloc<double>(std::max(dN, 1LL));
        if (G->nfree > 0) {
            int nr = G->d + G->rot();
            Xf = dalloc<T>((size_t)nr * std::max(dN, 1LL));
            Nb = dalloc<double>((size_t)G->nfree * nr * nr);
            rU = dalloc<double>(G->nU);
            sU = dalloc<double>(G->nU);
            Uo = dalloc<double>(G->nU);
        }
    }

    // X = M~^-1 K_f column by column, then the body blocks K_f^T X and their
    // FP64 inverses (the free bodies' mobilities, Sec. VIII)
    void setup_free() {
        if (G->nfree == 0 || free_ready) return;
        cudaStream_t s = G->stream;
        int d = G->d, nr = d + G->rot(), N = G->N, B = (int)G->bodies.size();
        long long dN = (long long)N * d;
        double* col = nullptr;
        double* unit = nullptr;
        T* colT = nullptr;
        IBR_CUDA_TRY(cudaMallocAsync(&col, sizeof(double) * dN, s));
        IBR_CUDA_TRY(cudaMallocAsync(&unit, sizeof(double) * G->nU, s));
        IBR_CUDA_TRY(cudaMallocAsync(&colT, sizeof(T) * dN, s));
        std::vector<double> hu(G->nU);
        std::vector<double> hN((size_t)G->nfree * nr * nr);
        std::vector<double> kt(G->nU);
        for (int c = 0; c < nr; ++c) {
            for (int fb = 0; fb < G->nfree; ++fb)
                for (int q = 0; q < nr; ++q) hu[fb * nr + q] = q == c ? 1.0 : 0.0;
            IBR_CUDA_TRY(cudaMemcpyAsync(unit, hu.data(), sizeof(double) * G->nU, cudaMemcpyHostToDevice, s));
            IBR_CUDA_TRY(cudaMemsetAsync(col, 0, sizeof(double) * dN, s));
            rigid_K_free(d, N, G->md.rel, G->md.body, G->bfree_dev, unit, col, 1.0, s);
            vec_convert<double, T>(dN, col, colT, s);
            blockdiag_gemv<T, T>(G->nblk, G->moff_dev, G->roff_dev, (int)dN, Minv, colT, Xf + (long long)c * dN, s);
            rigid_KT_free<T>(d, B, G->md.body_start, G->bfree_dev, G->md.rel, Xf + (long long)c * dN, sU, s);
            IBR_CUDA_TRY(cudaMemcpyAsync(kt.data(), sU, sizeof(double) * G->nU, cudaMemcpyDeviceToHost, s));
            IBR_CUDA_TRY(cudaStreamSynchronize(s));
            for (int fb = 0; fb < G->nfree; ++fb)
                for (int q = 0; q < nr; ++q) hN[((size_t)fb * nr + q) * nr + c] = kt[fb * nr + q];
        }
        IBR_CUDA_TRY(cudaMemcpyAsync(Nb, hN.data(), sizeof(double) * hN.size(), cudaMemcpyHostToDevice, s));
        IBR_CUDA_TRY(cudaMemsetAsync(G->info_dev, 0, sizeof(int), s));
        small_inverse(G->nfree, nr, Nb, G->info_dev, s);
        int info = 0;
        IBR_CUDA_TRY(cudaMemcpyAsync(&info, G->info_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
        IBR_CUDA_TRY(cudaStreamSynchronize(s));
        cudaFree(col);
        cudaFree(unit);
        cudaFree(colT);
        if (info) throw Error{IBR_ENUMERIC, "a free body's resistance block K^T M~^-1 K is singular"};
        free_ready = true;
    }
    ~PC() {
        invalidate_graph();
        dfree(rL);
        dfree(Xf);
        dfree(Nb);
        dfree(rU);
        dfree(sU);
        dfree(Uo);
        mg.release();
        T* tp[] = {Vi, Zi, w, rs, rs2, xs, y, phi, q, qr, dU, lamT};
        for (T* p : tp)
            if (p) cudaFree(p);
        double* dp[] = {Hi, cs, sn, gv, yv, h1, h2, sc, partial, means, shift, hk2, st};
        for (double* p : dp)
            if (p) cudaFree(p);
    }

    // z = P_S^-1 r (Sec. V.B, Eq. P1_practical)
    void apply_ps(const T* in, T* out) {
        cudaStream_t s = G->stream;
        const Geo& g = G->geo;
        long long n = g.ncell;
        int d = G->d;
        double sigma = G->sigma();
        mg.vcycle(y, in, d, 0, sigma, G->eta, true, pre, post, s);              // y = A~^-1 g
        ps_divergence<T>(g, y, in + d * n, qr, -1.0 / (g.h * g.h), q, s);      // q = -D y - h
        mg.vcycle(phi, qr, 1, FLD_P, 0.0, 1.0, true, pre, post, s);             // phi = L~p^-1 q
        double cphi = G->steady() ? 0.0 : -G->rho * g.h * g.h / G->dt;
        ps_finish<T>(g, y, phi, q, out, G->eta, cphi, s);                       // v, pi
        ++ps_count;
    }

    // x = GMRES(ns) approximation of [A G; -D 0]^-1 rhs, x0 = 0
    void inner_gmres(const T* rhs, T* xout) {
        cudaStream_t s = G->stream;
        const Geo& g = G->geo;
        long long nS = G->nS;
        norm2<T>(nS, rhs, partial, sc + 0, s);
        givens_init(sc + 0, gv, ns + 1, sc + 1, sc + 2, s);
        scale_rsqrt<T, T>(nS, sc + 2, rhs, Vi, nullptr, 0, s);
        for (int j = 0; j < ns; ++j) {
            T* Vj = Vi + (long long)j * nS;
            T* Zj = Zi + (long long)j * nS;
            apply_ps(Vj, Zj);
            stokes_apply<T>(g, Zj, w, G->sigma(), G->eta, nullptr, s);
            // the last step only needs its Hessenberg column (the inner solve is
            // a preconditioner: one Gram-Schmidt pass, the norm from |w|^2 - |h|^2)
            if (j + 1 < ns)
                cgs_orthonormalize<T, T>(nS, Vi, nS, j + 1, w, Vi + (long long)(j + 1) * nS, nullptr, 0, partial, h1,
                                         h2, hk2, st, s);
            else
                cgs_coeffs_only<T>(nS, Vi, nS, j + 1, w, partial, h1, h2, st, s);
            arnoldi_column(Hi, ns + 1, h1, h2, st + 2, j, cs, sn, gv, sc + 3, sc + 4, s);
        }
        hess_solve(Hi, ns + 1, gv, ns, yv, s);
        combine<T, T>(nS, Zi, nS, ns, yv, xout, false, s);
    }

    // z = P^-1 r for the constrained system (Sec. V.A), FP64 in and out
    // steps 1-4 of Sec. V.A from rs (fluid part, precision T) and rL (the
    // constraint part, FP64) into xs (v, pi) and lamT (Lambda); fixed buffers
    // only, so the whole sequence can be captured as one CUDA graph
    void body() {
        cudaStream_t s = G->stream;
        const Geo& g = G->geo;
        long long n = g.ncell, nS = G->nS;
        int d = G->d, N = G->N;
        long long dN = (long long)N * d;
        inner_gmres(rs, xs);                                                 // step 1
        if (N > 0) {
            interp<T, double>(g, G->md, xs, dU, -1.0, rL, s, -1.0);          // step 2: dU = -(J v + W)
            blockdiag_gemv<T, T>(G->nblk, G->moff_dev, G->roff_dev, (int)dN, Minv, dU, lamT,
                                 s);                                        // step 3
            if (G->nfree > 0) {
                // free bodies: [M~ -K_f; K_f^T 0][Lambda; U] = [dU; F]  ->
                // U = N (F - K_f^T M~^-1 dU), Lambda = M~^-1 dU + X U
                rigid_KT_free<T>(d, (int)G->bodies.size(), G->md.body_start, G->bfree_dev, G->md.rel, lamT, sU, s);
                body_solve(G->nfree, d + G->rot(), Nb, rU, sU, Uo, s);
                lam_add_XU<T>(d, N, G->md.body, G->bfree_dev, Xf, Uo, lamT, s);
            }
            if (variant == IBR_PC_FULL) {                                   // step 4
                IBR_CUDA_TRY(cudaMemcpyAsync(rs2, rs, sizeof(T) * nS, cudaMemcpyDeviceToDevice, s));
                spread_gather<T>(G->md, lamT, rs2, 1.0 / std::pow(g.h, d), s);
                if (G->null_v()) {
                    lam_sum<T>(d, N, lamT, 1.0 / G->vol, shift, s);
                    subtract_means<T>(n, d, rs2, shift, s);
                }
                inner_gmres(rs2, xs);
            }
        }
        // keep the Krylov vectors in the space of the constrained problem:
        // <v> = 0 (periodic steady Stokes) and <pi> = 0
        block_means<T>(n, d + 1, xs, partial, means, s);
        if (G->null_v())
            subtract_means<T>(n, d + 1, xs, means, s);
        else
            subtract_means<T>(n, 1, xs + (long long)d * n, means + d, s);
    }

    static bool use_graphs() {
        static const bool off = [] {
            const char* e = std::getenv("IBR_GRAPHS");
            return e && e[0] == '0';
        }();
        return !off && !profiling_enabled();
    }

    // z = P^-1 r for the constrained system (Sec. V.A), FP64 in and out.
    // fluid_prepared: rs already holds r's fluid part in precision T.
    void apply(const double* r, double* z, bool fluid_prepared = false) {
        cudaStream_t s = G->stream;
        long long nS = G->nS;
        int N = G->N;
        long long dN = (long long)N * G->d;
        if (!fluid_prepared) vec_convert<double, T>(nS, r, rs, s);
        if (N > 0) IBR_CUDA_TRY(cudaMemcpyAsync(rL, r + nS, sizeof(double) * dN, cudaMemcpyDeviceToDevice, s));
        if (G->nfree > 0)
            IBR_CUDA_TRY(cudaMemcpyAsync(rU, r + nS + dN, sizeof(double) * G->nU, cudaMemcpyDeviceToDevice, s));
        long long ps_per = (long long)ns * (variant == IBR_PC_FULL && N > 0 ? 2 : 1);
        if (use_graphs()) {
            if (gexec && (g_ns != ns || g_pre != pre || g_post != post || g_variant != variant)) invalidate_graph();
            if (!gexec) {
                long long l0 = thread_launches();
                long long psc = ps_count;
                cudaGraph_t graph = nullptr;
                IBR_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
                try {
                    body();
                } catch (...) {
                    cudaStreamEndCapture(s, &graph);
                    if (graph) cudaGraphDestroy(graph);
                    throw;
                }
                IBR_CUDA_TRY(cudaStreamEndCapture(s, &graph));
                cudaError_t e = cudaGraphInstantiate(&gexec, graph, 0);
                cudaGraphDestroy(graph);
                IBR_CUDA_TRY(e);
                g_ns = ns;
                g_pre = pre;
                g_post = post;
                g_variant = variant;
                g_launches = thread_launches() - l0;
                add_launches(-g_launches);  // counted again on every replay below
                ps_count = psc;
            }
            IBR_CUDA_TRY(cudaGraphLaunch(gexec, s));
            add_launches(g_launches);
            ps_count += ps_per;
        } else {
            body();
        }
        vec_convert<T, double>(nS, xs, z, s);
        if (N > 0) vec_convert<T, double>(dN, lamT, z + nS, s);
        if (G->nfree > 0)
            IBR_CUDA_TRY(cudaMemcpyAsync(z + nS + dN, Uo, sizeof(double) * G->nU, cudaMemcpyDeviceToDevice, s));
    }
};

namespace {

void require(bool c, const std::string& msg) {
    if (!c) throw Error{IBR_EINVAL, msg};
}

void quat_to_R(const double* q, double* R) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double nrm = std::sqrt(w * w + x * x + y * y + z * z);
    require(nrm > 0, "quaternion must be nonzero");
    w /= nrm;
    x /= nrm;
    y /= nrm;
    z /= nrm;
    R[0] = 1 - 2 * (y * y + z * z);
    R[1] = 2 * (x * y - w * z);
    R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);
    R[4] = 1 - 2 * (x * x + z * z);
    R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);
    R[7] = 2 * (y * z + w * x);
    R[8] = 1 - 2 * (x * x + y * y);
}

void free_markers(ibr_grid* G) {
    MarkerData& md = G->md;
    dfree(md.q);
    dfree(md.rel);
    dfree(md.body);
    dfree(md.body_start);
    dfree(md.idx);
    dfree(md.w64);
    dfree(md.w32);
    dfree(md.face);
    dfree(md.off);
    dfree(md.ent_m);
    dfree(md.ent_w64);
    dfree(md.ent_w32);
    md.F = md.E = 0;
    dfree(G->moff_dev);
    dfree(G->roff_dev);
    dfree(G->Mbuild);
    dfree(G->Minv64);
    dfree(G->Minv32);
    dfree(G->FT);
    dfree(G->UO);
    dfree(G->bfree_dev);
}

void free_outer(ibr_grid* G) {
    double** ps[] = {&G->V, &G->Z, &G->b, &G->x, &G->w, &G->H, &G->cs, &G->sn, &G->gv, &G->yv,
                     &G->h1, &G->h2, &G->sc, &G->partial, &G->shift, &G->means, &G->hk2, &G->st, &G->vk64};
    for (double** p : ps) dfree(*p);
    dfree(G->wait_err);
    G->m_alloc = 0;
    G->have_solution = false;  // x is gone
}

// fill default options
void opts_default(ibr_solve_opts* o) {
    std::memset(o, 0, sizeof(*o));
    o->tol = 1e-8;
    o->restart = 50;
    o->max_iters = 1000;
    o->n_s = 0;  // automatic: 2 on periodic grids, 4 with walls
    o->variant = IBR_PC_LOWER;
    o->mg_pre = 2;
    o->mg_post = 2;
    o->mob_model = IBR_MOB_AUTO;
    o->mob_a_over_h = 0.0;            // the kernel's value (ibr_mobility_defaults)
    for (double& c : o->mob_coef) c = 0.0;  // all zero: the kernel's fitted App. B set
    o->time_cap_ms = 0.0;
}

// self-mobility f(0), the diagonal of M~ (Sec. IV.B): RPY (6 pi eta a)^-1
// minus the periodic correction, or the App. B value ln(l/(3.708 a))/(4 pi eta)
double mob_self(const MobParams& p) {
    if (p.model == IBR_MOB_RPY) return 1.0 / (6.0 * M_PI * p.eta * p.a) - p.corr;
    return std::log(p.l / (3.708 * p.a)) / (4.0 * M_PI * p.eta);
}

// The library's 2-D steady M~ (App. B, Eq. fg_steady_2d) per kernel: the
// coefficients a0..a4, b0..b3 of the rational forms and the marker radius a/h
// of the self-mobility f(0) = ln(l / (3.708 a)) / (4 pi eta), fitted by the
// paper's procedure (Sec. IV.B, App. B) to the library's own periodic pair
// mobility on a 256^2 grid (fit_mobility_2d.py; its output is
// mobility_fit_2d.json beside this package: rms error 0.003 in f~, 0.006 in g~
// over 0.1 <= r/h <= 20)
constexpr double AOH_2D_PESKIN4 = 1.0427568763030746;
constexpr double AOH_2D_BKP6 = 1.2268447983609203;
constexpr double COEF_2D_PESKIN4[9] = {0.4285760175890488, 0.07516239469333616, 0.15497843271654263,
                                       0.2490767399813471, 0.14442948562926494, 0.17060454818657458,
                                       0.09800169052231841, 4.121975016785502e-14, 0.18362839492192692};
constexpr double COEF_2D_BKP6[9] = {0.31867428077511517, 0.029809829931491737, 0.09128850757187502,
                                    0.21765971572545198, 0.10879540295508049, 0.13289304886387499,
                                    0.055576820005161384, 2.9295447563918447e-15, 0.14216790154120185};

MobParams mob_params(const ibr_grid* G, const ibr_solve_opts& o) {
    MobParams p;
    std::memset(&p, 0, sizeof(p));
    int model = o.mob_model & ~IBR_MOB_COUPLED;
    if (model == IBR_MOB_AUTO) model = G->d == 3 ? IBR_MOB_RPY : IBR_MOB_FIT2D;
    require(model == IBR_MOB_RPY || model == IBR_MOB_FIT2D, "unknown mob_model");
    require(!(model == IBR_MOB_FIT2D && G->d != 2), "IBR_MOB_FIT2D is a 2-D model");
    require(!(model == IBR_MOB_RPY && G->d != 3), "IBR_MOB_RPY is a 3-D model");
    // default marker radius: in 3-D a = 1.25 h for the 4-point kernel and
    // 1.47 h for the six-point kernel (Sec. IV.A); in 2-D the value at which
    // ln(l/(3.708 a))/(4 pi eta) equals the kernel's discrete periodic
    // self-mobility (App. B)
    const bool six = G->geo.kw == 6;
    double aoh = o.mob_a_over_h > 0 ? o.mob_a_over_h
                                    : (model == IBR_MOB_RPY ? (six ? 1.47 : 1.25) : (six ? AOH_2D_BKP6 : AOH_2D_PESKIN4));
    p.model = model;
    p.eta = G->eta;
    p.h = G->h;
    // the length in the 2-D self-mobility: the box (periodic), or the
    // narrowest wall-bounded extent (walls screen the logarithmic growth)
    p.l = G->L[0];
    if (G->walls()) {
        p.l = 1e300;
        for (int a = 0; a < G->d; ++a)
            if ((G->geo.wall >> a) & 1) p.l = std::min(p.l, G->L[a]);
    }
    p.a = aoh * G->h;
    for (int a = 0; a < 3; ++a) p.box[a] = (a < G->d && !((G->geo.wall >> a) & 1)) ? G->L[a] : 0.0;
    // periodic-image correction of App. A (fully periodic boxes only)
    p.corr = (model == IBR_MOB_RPY && !G->walls()) ? 2.84 / (6.0 * M_PI * G->eta * G->L[0]) : 0.0;
    bool zero = true;
    for (double c : o.mob_coef) zero = zero && c == 0.0;
    if (zero)
        std::memcpy(p.coef, six ? COEF_2D_BKP6 : COEF_2D_PESKIN4, sizeof(p.coef));
    else
        std::memcpy(p.coef, o.mob_coef, sizeof(p.coef));
    return p;
}

void ensure_pc(ibr_grid* G, int ns) {
    if (G->precision == IBR_FP64) {
        if (G->pc64 && G->pc_ns >= ns) return;
        delete G->pc64;
        G->pc64 = nullptr;
        G->pc64 = new PC<double>(G, ns);
    } else {
        if (G->pc32 && G->pc_ns >= ns) return;
        delete G->pc32;
        G->pc32 = nullptr;
        G->pc32 = new PC<float>(G, ns);
    }
    G->pc_ns = ns;
}

// The true mobility M0 = J L^-1 S (Sec. III.C: the Schur complement of the
// constrained system) into M0 (dN x dN, row-major, symmetrised), one column
// per marker force component: spread the unit force, solve the unconstrained
// Stokes problem by restarted GMRES(30) with P_S in FP64 to a relative
// residual of 1e-8, interpolate.  Returns the mean diagonal entry (the
// self-mobility scale used by the factorisation's pivot test).
double build_true_mobility(ibr_grid* G, double* M0) {
    cudaStream_t s = G->stream;
    const Geo& g = G->geo;
    const int d = G->d, N = G->N;
    const long long n = g.ncell, nS = G->nS, dN = (long long)N * d;
    PC<double> pc(G, 30);
    double* ek = dalloc<double>(dN);
    double* rhs = dalloc<double>(nS);
    double* x = dalloc<double>(nS);
    double* w = dalloc<double>(nS);
    double* dx = dalloc<double>(nS);
    double* hs = nullptr;
    IBR_CUDA_TRY(cudaMallocHost(&hs, 2 * sizeof(double)));
    auto norm_sq = [&](const double* v) {
        norm2<double>(nS, v, pc.partial, pc.sc, s);
        IBR_CUDA_TRY(cudaMemcpyAsync(hs, pc.sc, sizeof(double), cudaMemcpyDeviceToHost, s));
        IBR_CUDA_TRY(cudaStreamSynchronize(s));
        return hs[0];
    };
    hs[1] = 1.0;
    const double sc = 1.0 / std::pow(g.h, d);
    for (long long k = 0; k < dN; ++k) {
        IBR_CUDA_TRY(cudaMemsetAsync(ek, 0, sizeof(double) * dN, s));
        IBR_CUDA_TRY(cudaMemcpyAsync(ek + k, hs + 1, sizeof(double), cudaMemcpyHostToDevice, s));
        IBR_CUDA_TRY(cudaMemsetAsync(rhs, 0, sizeof(double) * nS, s));
        spread_gather<double>(G->md, ek, rhs, sc, s);
        if (G->null_v()) {
            lam_sum<double>(d, N, ek, 1.0 / G->vol, pc.shift, s);
            subtract_means<double>(n, d, rhs, pc.shift, s);
        }
        const double b2 = norm_sq(rhs);
        pc.inner_gmres(rhs, x);
        for (int pass = 1; pass < 8 && b2 > 0.0; ++pass) {
            stokes_apply<double>(g, x, w, G->sigma(), G->eta, nullptr, s);
            vec_axpby<double>(nS, 1.0, rhs, -1.0, w, s);  // w = rhs - L x
            if (norm_sq(w) <= 1e-16 * b2) break;
            pc.inner_gmres(w, dx);
            vec_axpby<double>(nS, 1.0, dx, 1.0, x, s);
        }
        if (G->null_v()) {
            block_means<double>(n, d, x, pc.partial, pc.means, s);
            subtract_means<double>(n, d, x, pc.means, s);
        }
        interp<double, double>(g, G->md, x, M0 + k * dN, 1.0, nullptr, s, 0.0);
    }
    std::vector<double> hM((size_t)dN * dN);
    IBR_CUDA_TRY(cudaMemcpyAsync(hM.data(), M0, hM.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    IBR_CUDA_TRY(cudaStreamSynchronize(s));
    double diag = 0.0;
    for (long long i = 0; i < dN; ++i) {
        diag += hM[(size_t)i * dN + i];
        for (long long j = i + 1; j < dN; ++j) {
            double a = 0.5 * (hM[(size_t)i * dN + j] + hM[(size_t)j * dN + i]);
            hM[(size_t)i * dN + j] = hM[(size_t)j * dN + i] = a;
        }
    }
    IBR_CUDA_TRY(cudaMemcpyAsync(M0, hM.data(), hM.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    IBR_CUDA_TRY(cudaStreamSynchronize(s));
    cudaFreeHost(hs);
    dfree(ek);
    dfree(rhs);
    dfree(x);
    dfree(w);
    dfree(dx);
    return diag / (double)dN;
}

// The pair-mobility table of IBR_MOB_PAIR: for each of PAIR_S source points
// x0 (off the grid nodes, in different sub-cell positions) and direction
// beta, v = L^-1 S~ e_beta delta(x - x0) by restarted GMRES(PAIR_NS) with
// P_S in FP64 to a relative residual of 1e-9, stored in FP32.  The pair
// mobility of two markers is approximately a function of their displacement
// only (Sec. IV: the kernel is close to translation invariant), so
// J(x0 + q_i - q_j) v is M_ij up to that (small) dependence on the sub-cell
// position, which the average over the source points reduces.
// Pair tables are shared by all grids of one shape (device, cells, box,
// eta, rho, dt, kernel): the first grid that needs one builds it, grids created
// later (e.g. several resident grids of a serving engine) reuse it; it is
// freed with the last grid that holds it.
struct PairTable {
    std::mutex mu;  // held while the table is built
    float* tab = nullptr;
    double* x0 = nullptr;
    ~PairTable() {
        if (tab) cudaFree(tab);
        if (x0) cudaFree(x0);
    }
};
std::mutex g_pair_mu;
std::map<std::string, std::weak_ptr<PairTable>> g_pair_cache;

std::string pair_key(const ibr_grid* G) {
    int dev = 0;
    cudaGetDevice(&dev);
    char buf[256];
    std::snprintf(buf, sizeof(buf), "%d|%d|%d,%d,%d|%.17g,%.17g,%.17g|%.17g|%.17g|%.17g|k%d", dev, G->d, G->n[0],
                  G->n[1], G->n[2], G->L[0], G->L[1], G->L[2], G->eta, G->rho, G->dt, G->geo.kw);
    return buf;
}

void build_pair_table_into(ibr_grid* G, float*& tab_out, double*& x0_out);

void build_pair_table(ibr_grid* G) {
    if (G->pair_tab) return;
    std::shared_ptr<PairTable> t;
    {
        std::lock_guard<std::mutex> lk(g_pair_mu);
        const std::string key = pair_key(G);
        t = g_pair_cache[key].lock();
        if (!t) {
            t = std::make_shared<PairTable>();
            g_pair_cache[key] = t;
        }
        for (auto it = g_pair_cache.begin(); it != g_pair_cache.end();)  // drop expired entries
            it = it->second.expired() ? g_pair_cache.erase(it) : std::next(it);
    }
    {
        std::lock_guard<std::mutex> lk(t->mu);
        if (!t->tab) build_pair_table_into(G, t->tab, t->x0);
    }
    G->pair_tab = t->tab;
    G->pair_x0 = t->x0;
    G->pair_hold = t;
}

void build_pair_table_into(ibr_grid* G, float*& tab_out, double*& x0_out) {
    cudaStream_t s = G->stream;
    const Geo& g = G->geo;
    const int d = G->d;
    const long long n = g.ncell, nS = G->nS;
    // sub-cell offsets of the sources (fractions of h), placed near the box centre
    const double frac[PAIR_S][3] = {{0.3, 0.7, 0.45}, {0.7, 0.3, 0.55}};
    double hx0[PAIR_S * 3];
    for (int k = 0; k < PAIR_S; ++k)
        for (int a = 0; a < d; ++a) hx0[k * d + a] = (std::floor(0.5 * G->n[a]) + frac[k][a]) * g.h;
    float* tab = dalloc<float>((size_t)PAIR_S * d * d * n);
    double* x0 = dalloc<double>((size_t)PAIR_S * d);
    PC<double> pc(G, PAIR_NS);
    double* rhs = dalloc<double>(nS);
    double* x = dalloc<double>(nS);
    double* w = dalloc<double>(nS);
    double* dx = dalloc<double>(nS);
    double* hs = nullptr;
    auto cleanup = [&] {
        dfree(rhs);
        dfree(x);
        dfree(w);
        dfree(dx);
        if (hs) cudaFreeHost(hs);
        hs = nullptr;
    };
    try {
        IBR_CUDA_TRY(cudaMallocHost(&hs, sizeof(double)));
        IBR_CUDA_TRY(cudaMemcpyAsync(x0, hx0, sizeof(double) * PAIR_S * d, cudaMemcpyHostToDevice, s));
        auto norm_sq = [&](const double* v) {
            norm2<double>(nS, v, pc.partial, pc.sc, s);
            IBR_CUDA_TRY(cudaMemcpyAsync(hs, pc.sc, sizeof(double), cudaMemcpyDeviceToHost, s));
            IBR_CUDA_TRY(cudaStreamSynchronize(s));
            return hs[0];
        };
        for (int k = 0; k < PAIR_S; ++k)
            for (int be = 0; be < d; ++be) {
                IBR_CUDA_TRY(cudaMemsetAsync(rhs, 0, sizeof(double) * nS, s));
                point_spread(g, x0 + k * d, be, 1.0 / std::pow(g.h, d), rhs, s);
                if (G->null_v()) {  // S~ = S - vol^-1 1^T: the force field has zero mean
                    block_means<double>(n, d, rhs, pc.partial, pc.means, s);
                    subtract_means<double>(n, d, rhs, pc.means, s);
                }
                const double b2 = norm_sq(rhs);
                IBR_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * nS, s));
                IBR_CUDA_TRY(cudaMemcpyAsync(w, rhs, sizeof(double) * nS, cudaMemcpyDeviceToDevice, s));
                for (int pass = 0; pass < 40; ++pass) {
                    pc.inner_gmres(w, dx);
                    vec_axpby<double>(nS, 1.0, dx, 1.0, x, s);
                    stokes_apply<double>(g, x, w, G->sigma(), G->eta, nullptr, s);
                    vec_axpby<double>(nS, 1.0, rhs, -1.0, w, s);  // w = rhs - L x
                    if (G->null_v()) {
                        block_means<double>(n, d + 1, w, pc.partial, pc.means, s);
                        subtract_means<double>(n, d + 1, w, pc.means, s);
                    }
                    if (norm_sq(w) <= 1e-18 * b2) break;
                }
                if (G->null_v()) {
                    block_means<double>(n, d, x, pc.partial, pc.means, s);
                    subtract_means<double>(n, d, x, pc.means, s);
                }
                vec_convert<double, float>((long long)d * n, x, tab + (size_t)(k * d + be) * d * n, s);
            }
        IBR_CUDA_TRY(cudaStreamSynchronize(s));
    } catch (...) {
        cleanup();
        dfree(tab);
        dfree(x0);
        throw;
    }
    cleanup();
    tab_out = tab;
    x0_out = x0;
}

void prepare(ibr_grid* G, const ibr_solve_opts& o) {
    cudaStream_t s = G->stream;
    require(!G->bodies.empty(), "no bodies added");
    int d = G->d;
    int B = (int)G->bodies.size();
    int N = 0;
    for (auto& b : G->bodies) {
        require(b.N > 0, "every body needs markers (ibr_set_markers)");
        N += b.N;
    }
    free_markers(G);
    G->N = N;
    G->md.N = N;
    G->md.B = B;
    G->bfree.assign(B, -1);
    G->nfree = 0;
    for (int bi = 0; bi < B; ++bi)
        if (G->bodies[bi].kin == IBR_FREE) G->bfree[bi] = G->nfree++;
    G->nU = G->nfree * (d + G->rot());
    G->len = G->nS + (long long)N * d + G->nU;
    std::vector<double> rb((size_t)N * d);
    std::vector<int> body(N), bstart(B + 1);
    std::vector<double> xcR((size_t)B * 12);
    int k = 0;
    for (int bi = 0; bi < B; ++bi) {
        const Body& b = G->bodies[bi];
        bstart[bi] = k;
        std::memcpy(&rb[(size_t)k * d], b.rbody.data(), sizeof(double) * b.N * d);
        for (int i = 0; i < b.N; ++i) body[k + i] = bi;
        k += b.N;
        for (int a = 0; a < 3; ++a) xcR[bi * 12 + a] = b.xc[a];
        for (int a = 0; a < 9; ++a) xcR[bi * 12 + 3 + a] = b.R[a];
    }
    bstart[B] = N;
    // markers on wall axes: inside the box, and outside the kernel support
    // (2h) of walls that carry nonzero boundary data (J_0 c is not formed)
    if (G->walls()) {
        bool data[6];
        for (int f = 0; f < 2 * d; ++f) {
            data[f] = false;
            for (double v : G->wdata_host[f]) data[f] = data[f] || v != 0.0;
        }
        const double tol = 1e-12 * G->h;
        for (int i = 0; i < N; ++i) {
            const double* P = &xcR[(size_t)body[i] * 12];
            const double* r = &rb[(size_t)i * d];
            for (int a = 0; a < d; ++a) {
                if (!((G->geo.wall >> a) & 1)) continue;
                double q = P[a];
                for (int e = 0; e < d; ++e) q += P[3 + 3 * a + e] * r[e];
                require(q >= -tol && q <= G->L[a] + tol, "a marker lies outside the walls");
                require(!(data[2 * a] && q < 2.0 * G->h - tol) && !(data[2 * a + 1] && q > G->L[a] - 2.0 * G->h + tol),
                        "a marker lies within the kernel support (2h) of a wall with nonzero boundary velocity");
            }
        }
    }
    MarkerData& md = G->md;
    double* rb_dev = dalloc<double>(rb.size());
    double* xcR_dev = dalloc<double>(xcR.size());
    md.q = dalloc<double>((size_t)N * d);
    md.rel = dalloc<double>((size_t)N * d);
    md.body = dalloc<int>(N);
    md.body_start = dalloc<int>(B + 1);
    const int kw = G->geo.kw;
    md.idx = dalloc<int>((size_t)N * d * d * kw);
    md.w64 = dalloc<double>((size_t)N * d * d * kw);
    md.w32 = dalloc<float>((size_t)N * d * d * kw);
    IBR_CUDA_TRY(cudaMemcpyAsync(rb_dev, rb.data(), rb.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    IBR_CUDA_TRY(cudaMemcpyAsync(xcR_dev, xcR.data(), xcR.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    IBR_CUDA_TRY(cudaMemcpyAsync(md.body, body.data(), body.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    IBR_CUDA_TRY(cudaMemcpyAsync(md.body_start, bstart.data(), bstart.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    double Lwrap[3] = {0.0, 0.0, 0.0};  // periodic axes wrap, wall axes do not
    for (int a = 0; a < d; ++a) Lwrap[a] = ((G->geo.wall >> a) & 1) ? 0.0 : G->L[a];
    markers_positions(d, N, rb_dev, md.body, xcR_dev, Lwrap, md.q, md.rel, s);
    markers_weights(G->geo, N, md.q, md.idx, md.w64, md.w32, s);
    markers_build_gather(G->geo, md, s);
    // the Schur-complement approximation: the analytic M~, one dense block per
    // body (Sec. IV, VIII), or the true mobility M0 = J L^-1 S of all markers
    // as one block, computed from the library's own Stokes solves (Sec. V.C:
    // worth it for fixed geometries, e.g. the steady nozzle of Sec. VII.F)
    const bool true_mob = o.mob_model == IBR_MOB_TRUE;
    const bool pair_mob = o.mob_model == IBR_MOB_PAIR;
    require(!(pair_mob && G->walls()), "IBR_MOB_PAIR needs a periodic grid");
    // the pair table, and the analytic forms with IBR_MOB_COUPLED, couple all
    // bodies in one block (M~_ij for every marker pair, Sec. IV.B) while
    // d N <= pair_full_max(); otherwise one block per body (the block-diagonal
    // form of Sec. IX, interactions between bodies left out)
    const bool coupled = pair_mob || (o.mob_model & IBR_MOB_COUPLED);
    const bool one_block = true_mob || (coupled && (long long)N * d <= pair_full_max());
    G->nblk = one_block ? 1 : B;
    const int nblk = G->nblk;
    G->moff.assign(nblk + 1, 0);
    G->roff.assign(nblk + 1, 0);
    for (int bi = 0; bi < nblk; ++bi) {
        long long nb = one_block ? (long long)N * d : (long long)G->bodies[bi].N * d;
        G->moff[bi + 1] = G->moff[bi] + nb * nb;
        G->roff[bi + 1] = G->roff[bi] + (int)nb;
    }
    G->moff_dev = dalloc<long long>(nblk + 1);
    G->roff_dev = dalloc<int>(nblk + 1);
    IBR_CUDA_TRY(cudaMemcpyAsync(G->moff_dev, G->moff.data(), (nblk + 1) * sizeof(long long), cudaMemcpyHostToDevice,
                                 s));
    IBR_CUDA_TRY(cudaMemcpyAsync(G->roff_dev, G->roff.data(), (nblk + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
    long long mtot = G->moff[nblk];
    G->Mbuild = dalloc<double>(mtot);
    double fself = 0.0;
    if (true_mob) {
        fself = build_true_mobility(G, G->Mbuild);
    } else if (pair_mob) {
        build_pair_table(G);
        for (int bi = 0; bi < nblk; ++bi) {
            const int m0 = one_block ? 0 : bstart[bi];
            const int nm = one_block ? N : G->bodies[bi].N;
            pair_mtilde(G->geo, nm, md.q + (long long)m0 * d, PAIR_S, G->pair_x0, G->pair_tab, G->Mbuild + G->moff[bi],
                        s);
        }
        // the self-mobility scale: mean of the first marker's diagonal entries
        const long long ld = G->roff[1] - G->roff[0];
        double dg[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < d; ++a)
            IBR_CUDA_TRY(cudaMemcpyAsync(&dg[a], G->Mbuild + a * ld + a, sizeof(double), cudaMemcpyDeviceToHost, s));
        IBR_CUDA_TRY(cudaStreamSynchronize(s));
        for (int a = 0; a < d; ++a) fself += dg[a] / d;
    } else {
        MobParams mp = mob_params(G, o);
        if (one_block)
            mtilde_build(d, N, md.q, mp, G->Mbuild, s);  // lab positions, minimum images
        else
            for (int bi = 0; bi < B; ++bi)
                mtilde_build(d, G->bodies[bi].N, md.rel + (long long)bstart[bi] * d, mp, G->Mbuild + G->moff[bi], s);
        fself = mob_self(mp);
    }
    // info_dev[0]: failed pivot, info_dev[1]: tensor-core time-out flag
    if (!G->info_dev) G->info_dev = dalloc<int>(2);
    IBR_CUDA_TRY(cudaMemsetAsync(G->info_dev, 0, 2 * sizeof(int), s));
    // a pivot below this fraction of the self-mobility means M~ is singular
    // to working precision (e.g. coincident markers)
    if (!(fself > 0.0))
        throw Error{IBR_ENUMERIC, "self-mobility f(0) of M~ is not positive (check mob_a_over_h, box size)"};
    double min_piv64 = 1e-10 * fself, min_piv32 = 1e-5 * fself;
    long long maxblk = 0;
    for (int bi = 0; bi < nblk; ++bi) maxblk = std::max(maxblk, G->moff[bi + 1] - G->moff[bi]);
    // Factor each block; if M~ is not positive definite (the analytic M~ need
    // not be, Sec. V.C) retry with M~ + delta I, delta growing geometrically
    // from 1e-3 f(0): the shift damps the spurious small/negative modes the way
    // the paper's eigenvalue filtering drops them.
    G->mob_shift.assign(nblk, 0.0);
    // the mixed path factorises on the tensor cores (split TF32); IBR_DENSE=cuda
    // selects the CUDA-core FP32 tiles instead (for comparison)
    static const bool dense_cuda = [] {
        const char* e = std::getenv("IBR_DENSE");
        return e && std::strcmp(e, "cuda") == 0;
    }();
    auto factor_all = [&](auto* Minv, auto* work, double min_piv) {
        using TT = std::remove_pointer_t<decltype(Minv)>;
        for (int bi = 0; bi < nblk; ++bi) {
            int nb = G->roff[bi + 1] - G->roff[bi];
            double delta = 0.0;
            for (int attempt = 0;; ++attempt) {
                mat_convert<double, TT>(G->moff[bi + 1] - G->moff[bi], G->Mbuild + G->moff[bi], Minv + G->moff[bi], s);
                if (delta > 0.0) add_diag<TT>(nb, Minv + G->moff[bi], delta, s);
                IBR_CUDA_TRY(cudaMemsetAsync(G->info_dev, 0, 2 * sizeof(int), s));
                if constexpr (std::is_same<TT, float>::value) {
                    if (!dense_cuda)
                        spd_inverse_tc(nb, Minv + G->moff[bi], G->info_dev, min_piv, fself, G->info_dev + 1, s);
                    else
                        spd_inverse<TT>(nb, Minv + G->moff[bi], work, G->info_dev, min_piv, s);
                } else {
                    spd_inverse<TT>(nb, Minv + G->moff[bi], work, G->info_dev, min_piv, s);
                }
                int info[2] = {0, 0};
                IBR_CUDA_TRY(cudaMemcpyAsync(info, G->info_dev, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
                IBR_CUDA_TRY(cudaStreamSynchronize(s));
                if (info[1]) throw Error{IBR_ECUDA, "a tensor-core product timed out waiting for its MMAs"};
                if (info[0] == 0) break;
                if (attempt >= 40)
                    throw Error{IBR_ENUMERIC, "mobility block " + std::to_string(bi) +
                                                  " could not be made positive definite"};
                delta = delta == 0.0 ? 1e-3 * fself : 2.0 * delta;
            }
            G->mob_shift[bi] = delta;
        }
    };
    if (G->precision == IBR_FP64) {
        G->Minv64 = dalloc<double>(mtot);
        double* work = dalloc<double>(maxblk);
        factor_all(G->Minv64, work, min_piv64);
        cudaFree(work);
    } else {
        G->Minv32 = dalloc<float>(mtot);
        float* work = dense_cuda ? dalloc<float>(maxblk) : nullptr;  // the tensor-core path has its own
        factor_all(G->Minv32, work, min_piv32);
        if (work) cudaFree(work);
    }
    G->FT = dalloc<double>((size_t)B * (d + G->rot()));
    G->bfree_dev = dalloc<int>(B);
    IBR_CUDA_TRY(cudaMemcpyAsync(G->bfree_dev, G->bfree.data(), B * sizeof(int), cudaMemcpyHostToDevice, s));
    G->UO = dalloc<double>((size_t)B * (d + G->rot()));
    cudaFree(rb_dev);
    cudaFree(xcR_dev);
    if (G->pc64) G->pc64->alloc_markers();
    if (G->pc32) G->pc32->alloc_markers();
    G->prepared_opts = o;
    G->dirty = false;
    G->have_solution = false;
}

bool mob_opts_equal(const ibr_solve_opts& a, const ibr_solve_opts& b) {
    return a.mob_model == b.mob_model && a.mob_a_over_h == b.mob_a_over_h &&
           std::memcmp(a.mob_coef, b.mob_coef, sizeof(a.mob_coef)) == 0;
}

void ensure_outer(ibr_grid* G, int m) {
    // the workspace is kept while it is large enough (a resident grid reused
    // with another marker count); w's zero pad entry moves with len
    if (G->m_alloc >= m && G->V && G->len_alloc >= G->len) {
        if (G->w_len != G->len) {
            IBR_CUDA_TRY(cudaMemsetAsync(G->w, 0, ((G->len_alloc + 1) & ~1LL) * sizeof(double), G->stream));
            // the basis columns now have the new length's stride: their pad
            // entries (read by the paired Gram-Schmidt passes) must be zero
            const long long lpn = G->len_pad();
            if (lpn > G->len)
                IBR_CUDA_TRY(cudaMemset2DAsync(G->V + G->len, lpn * sizeof(double), 0,
                                               (lpn - G->len) * sizeof(double), G->m_alloc + 1, G->stream));
            G->w_len = G->len;
        }
        return;
    }
    free_outer(G);
    long long len = G->len;
    G->w_len = len;
    // the double-float basis is read in pairs: an even leading dimension,
    // and w carries the same zero pad entry
    const long long lp = G->len_pad();
    G->V = dalloc<double>((size_t)(m + 1) * lp);
    // the Gram-Schmidt passes read whole entry pairs: a pad entry (odd len) is zero
    if (lp > len)
        IBR_CUDA_TRY(cudaMemset2DAsync(G->V + len, lp * sizeof(double), 0, (lp - len) * sizeof(double), m + 1,
                                       G->stream));
    G->vk64 = dalloc<double>(len);
    G->Z = dalloc<double>((size_t)m * len);
    G->b = dalloc<double>(len);
    G->x = dalloc<double>(len);
    G->w = dalloc<double>(lp);
    IBR_CUDA_TRY(cudaMemsetAsync(G->w, 0, lp * sizeof(double), G->stream));
    G->H = dalloc<double>((size_t)(m + 1) * (m + 1));
    G->cs = dalloc<double>(m + 1);
    G->sn = dalloc<double>(m + 1);
    G->gv = dalloc<double>(m + 2);
    G->yv = dalloc<double>(m + 1);
    G->h1 = dalloc<double>(m + 2);
    G->h2 = dalloc<double>(m + 1);
    G->hk2 = dalloc<double>(m + 2);
    G->st = dalloc<double>(4);
    G->sc = dalloc<double>(8);
    G->wait_err = dalloc<int>(1);
    IBR_CUDA_TRY(cudaMemsetAsync(G->wait_err, 0, sizeof(int), G->stream));
    G->partial = dalloc<double>((size_t)RED_BLOCKS * std::max(m + 1, 4));
    G->shift = dalloc<double>(4);
    G->means = dalloc<double>(4);
    G->len_alloc = len;
    if (!G->host_sc) IBR_CUDA_TRY(cudaMallocHost(&G->host_sc, 8 * sizeof(double)));
    G->m_alloc = m;
}

// y = (system matrix) x  (FP64)
void full_matvec(ibr_grid* G, const double* x, double* y) {
    cudaStream_t s = G->stream;
    const Geo& g = G->geo;
    int d = G->d;
    long long nS = G->nS;
    const double* lam = x + nS;
    const double* shift = nullptr;
    if (G->null_v() && G->N > 0) {
        lam_sum<double>(d, G->N, lam, 1.0 / G->vol, G->shift, s);  // -S~ = -S + vol^-1 1^T
        shift = G->shift;
    }
    stokes_apply<double>(g, x, y, G->sigma(), G->eta, shift, s);
    if (G->N > 0) {
        spread_gather<double>(G->md, lam, y, -1.0 / std::pow(g.h, d), s);
        interp<double, double>(g, G->md, x, y + nS, -1.0, nullptr, s, 0.0);
    }
    if (G->nfree > 0) {
        // free bodies: -J v + K_f U_f on their markers, and K_f^T Lambda
        long long dN = (long long)G->N * d;
        rigid_K_free(d, G->N, G->md.rel, G->md.body, G->bfree_dev, x + nS + dN, y + nS, 1.0, s);
        rigid_KT_free<double>(d, (int)G->bodies.size(), G->md.body_start, G->bfree_dev, G->md.rel, lam,
                              y + nS + dN, s);
    }
}

// fluid_prepared: the FP32 copy of r's fluid part is already in pc32->rs
void pc_apply(ibr_grid* G, const double* r, double* z, bool fluid_prepared) {
    if (G->precision == IBR_FP64)
        G->pc64->apply(r, z);
    else
        G->pc32->apply(r, z, fluid_prepared);
}

double read_scalar(ibr_grid* G, const double* dev) {
    IBR_CUDA_TRY(cudaMemcpyAsync(G->host_sc, dev, sizeof(double), cudaMemcpyDeviceToHost, G->stream));
    IBR_CUDA_TRY(cudaStreamSynchronize(G->stream));
    return G->host_sc[0];
}

void project_solution(ibr_grid* G, double* x) {
    cudaStream_t s = G->stream;
    long long n = G->geo.ncell;
    int d = G->d;
    block_means<double>(n, d + 1, x, G->partial, G->means, s);
    if (G->null_v())
        subtract_means<double>(n, d + 1, x, G->means, s);
    else
        subtract_means<double>(n, 1, x + (long long)d * n, G->means + d, s);
}

// The outer Arnoldi orthogonalisation, over the FP64 basis in both
// precisions.  Systems of at least ARN_MGS_MIN_LEN entries: modified
// Gram-Schmidt (two FP64 FMAs per entry and basis vector; on this part the
// FP64 pipe, not HBM, bounds these passes, and MGS halves their work).
// Smaller systems: classical Gram-Schmidt with reorthogonalisation (CGS2, four
// FMAs) pipelined on bulk copies, three launches per step instead of MGS's
// k + 2 (there the passes are short and launch latency decides).
// IBR_ARNOLDI in the environment forces one: "mgs", "cgs2", or "df" (CGS2 over
// a double-float basis: pairs of floats, a 48-bit significand, arithmetic on
// the FP32 pipe; for comparison).
enum { ARN_MGS = 0, ARN_CGS2 = 1, ARN_DF = 2 };
constexpr long long ARN_MGS_MIN_LEN = 2000000;
int arnoldi_kind(long long len) {
    static const int forced = [] {
        const char* e = std::getenv("IBR_ARNOLDI");
        if (e && std::string(e) == "mgs") return (int)ARN_MGS;
        if (e && std::string(e) == "cgs2") return (int)ARN_CGS2;
        if (e && std::string(e) == "df") return (int)ARN_DF;
        return -1;
    }();
    if (forced >= 0) return forced;
    return len >= ARN_MGS_MIN_LEN ? (int)ARN_MGS : (int)ARN_CGS2;
}

// warm: start from the x already in G->x (time stepping), else from x = 0
int fgmres(ibr_grid* G, const ibr_solve_opts& o, ibr_solve_info& info, bool warm = false) {
    cudaStream_t s = G->stream;
    long long len = G->len;
    int m = o.restart;
    double t0 = now_ms();
    norm2<double>(len, G->b, G->partial, G->sc + 0, s);
    double bnorm = std::sqrt(read_scalar(G, G->sc + 0));
    if (!warm) IBR_CUDA_TRY(cudaMemsetAsync(G->x, 0, len * sizeof(double), s));
    info.iters = 0;
    info.restarts = 0;
    if (!(bnorm > 0.0)) {
        if (std::isnan(bnorm)) throw Error{IBR_ENUMERIC, "right-hand side contains NaN/Inf"};
        if (warm) IBR_CUDA_TRY(cudaMemsetAsync(G->x, 0, len * sizeof(double), s));
        info.rel_res_est = info.rel_res_true = 0.0;
        return IBR_OK;
    }
    double target = o.tol * bnorm;
    // IBR_VERBOSE=1 prints the Arnoldi residual estimates and the true
    // residual at each restart to stderr (diagnostics only)
    const char* ve = std::getenv("IBR_VERBOSE");
    bool verbose = ve && ve[0] && ve[0] != '0';
    bool first = !warm;
    bool last_cycle_converged_est = false;
    int stalls = 0;
    double last_rn = 0.0;
    int status = IBR_OK;
    while (true) {
        // r = b - A x  (into w)
        if (first) {
            IBR_CUDA_TRY(cudaMemcpyAsync(G->w, G->b, len * sizeof(double), cudaMemcpyDeviceToDevice, s));
        } else {
            full_matvec(G, G->x, G->w);
            vec_axpby<double>(len, 1.0, G->b, -1.0, G->w, s);
        }
        norm2<double>(len, G->w, G->partial, G->sc + 0, s);
        double rn = std::sqrt(read_scalar(G, G->sc + 0));
        info.rel_res_true = rn / bnorm;
        if (verbose) std::fprintf(stderr, "[ibr] restart %d true rel res %.3e\n", info.restarts, rn / bnorm);
        if (std::isnan(rn)) throw Error{IBR_ENUMERIC, "NaN in the FGMRES residual"};
        if (rn <= target) break;
        // a cycle that ended on the Givens estimate but left the true residual
        // where it was has hit the attainable accuracy of FP64 for this
        // scaling: stop after three such cycles instead of spinning
        if (!first && last_cycle_converged_est) {
            stalls = (rn > 0.5 * last_rn) ? stalls + 1 : 0;
            if (stalls >= 3) {
                status = IBR_ENOTCONV;
                break;
            }
        }
        last_rn = rn;
        if (info.iters >= o.max_iters) {
            status = IBR_ENOTCONV;
            break;
        }
        if (o.time_cap_ms > 0 && now_ms() - t0 > o.time_cap_ms) {
            status = IBR_ETIMEOUT;
            break;
        }
        givens_init(G->sc + 0, G->gv, m + 1, G->sc + 1, G->sc + 2, s);
        // V_0 = r / |r|; in mixed precision the preconditioner's FP32 copy of
        // its fluid part is written by the same pass
        float* rs32 = G->precision == IBR_MIXED ? G->pc32->rs : nullptr;
        const long long lp = G->len_pad();
        const int arn = arnoldi_kind(len);
        const bool df = arn == ARN_DF;
        // double-float basis: the preconditioner reads the fluid part from
        // rs32 (mixed) or vk64 (FP64), the constraint part from vk64
        const long long from64 = rs32 ? G->nS : 0;
        dflt* Vd = reinterpret_cast<dflt*>(G->V);
        if (df) {
            scale_df(lp, len, G->sc + 2, G->w, Vd, rs32, G->nS, G->vk64, from64, s);
        } else if (rs32) {
            // over the padded length: V_0's pad entry is w's (zero)
            scale_rsqrt<double, float>(lp, G->sc + 2, G->w, G->V, rs32, G->nS, s);
        } else {
            scale_rsqrt<double, double>(lp, G->sc + 2, G->w, G->V, nullptr, 0, s);
        }
        int k = 0;
        last_cycle_converged_est = false;
        for (int j = 0; j < m; ++j) {
            double* Zj = G->Z + (long long)j * len;
            double* Vj = G->V + (long long)j * lp;
            pc_apply(G, df ? G->vk64 : Vj, Zj, true);
            full_matvec(G, Zj, G->w);
            // the FP64 basis: the preconditioner reads V_{j+1} itself (and, mixed,
            // the FP32 copy of its fluid part in rs32)
            if (arn == ARN_MGS) {
                mgs_orthonormalize(lp, G->V, lp, j + 1, G->w, Vj + lp, rs32, G->nS, G->partial, G->h1, G->st, s);
            } else {
                cgs_orthonormalize_pipe(df, lp, len, G->V, lp, j + 1, G->w, Vj + lp, rs32, G->nS,
                                        df ? G->vk64 : nullptr, from64, G->partial, G->h1, G->h2, G->hk2, G->st,
                                        G->wait_err, s);
            }
            arnoldi_column(G->H, m + 1, G->h1, arn == ARN_MGS ? nullptr : G->h2, G->st + 2, j, G->cs, G->sn, G->gv,
                           G->sc + 3, G->sc + 4, s);
            k = j + 1;
            info.iters++;
            double est = read_scalar(G, G->sc + 3);
            info.rel_res_est = est / bnorm;
            if (verbose) {
                double hn = std::sqrt(read_scalar(G, G->st + 2));
                double re = read_scalar(G, G->st + 1);
                std::fprintf(stderr, "[ibr] it %d j %d est %.3e |w_perp| %.3e reorth %d\n", info.iters, j,
                             est / bnorm, hn, (int)re);
            }
            if (std::isnan(est)) throw Error{IBR_ENUMERIC, "NaN in the FGMRES Arnoldi process"};
            if (est <= target) last_cycle_converged_est = true;
            if (est <= target || info.iters >= o.max_iters) break;
            if (o.time_cap_ms > 0 && now_ms() - t0 > o.time_cap_ms) break;
        }
        {
            // the pipelined Gram-Schmidt passes flag a wait that timed out
            int werr = 0;
            IBR_CUDA_TRY(cudaMemcpyAsync(&werr, G->wait_err, sizeof(int), cudaMemcpyDeviceToHost, s));
            IBR_CUDA_TRY(cudaStreamSynchronize(s));
            if (werr) throw Error{IBR_ECUDA, "a pipelined Gram-Schmidt pass timed out waiting for its copies"};
        }
        hess_solve(G->H, m + 1, G->gv, k, G->yv, s);
        combine<double, double>(len, G->Z, len, k, G->yv, G->x, true, s);
        project_solution(G, G->x);
        info.restarts++;
        first = false;
    }
    return status;
}

}  // namespace

namespace {
int run_guarded(const char* fn, const std::function<void()>& body) {
    try {
        body();
        ibr::set_error("");
        return IBR_OK;
    } catch (const Error& e) {
        ibr::set_error(std::string(fn) + ": " + e.msg);
        return e.code;
    } catch (const std::bad_alloc&) {
        ibr::set_error(std::string(fn) + ": host allocation failed");
        return IBR_ENOMEM;
    } catch (const std::exception& e) {
        ibr::set_error(std::string(fn) + ": " + e.what());
        return IBR_EINVAL;
    }
}
}  // namespace

// One solve of the constrained system: options checked, set-up on demand,
// b = [g + wall data; wall data; W = -K U; F], FGMRES (from x = 0, or from
// the current x when warm), wall faces set.  Returns the FGMRES status.
int solve_core(ibr_grid* G, const double* body_UO, const double* gforce, int g_on_device,
               const ibr_solve_opts* opts, ibr_solve_info& info, bool warm) {
    require(G && body_UO, "grid and body_UO must be non-NULL");
    ibr_solve_opts o;
    if (opts)
        o = *opts;
    else
        opts_default(&o);
    require(o.tol > 0 && o.tol < 1, "tol must be in (0,1)");
    require(o.restart >= 1 && o.restart <= 120, "restart must be in [1,120]");
    require(o.n_s >= 0 && o.n_s <= 16, "n_s must be in [0,16]");
    // N_s = 2 for periodic problems (Sec. VII.A); near no-slip walls the
    // projection preconditioner is further from the Stokes inverse and
    // N_s = 4 is the robust choice (Sec. VII.A)
    if (o.n_s == 0) o.n_s = G->walls() ? 4 : 2;
    require(o.max_iters >= 1, "max_iters must be >= 1");
    require(o.variant == IBR_PC_LOWER || o.variant == IBR_PC_FULL, "bad variant");
    require(o.mg_pre >= 0 && o.mg_post >= 0 && o.mg_pre + o.mg_post >= 1, "bad mg sweeps");
    cudaStream_t s = G->stream;
    double t0 = now_ms();
    if (G->dirty || !mob_opts_equal(o, G->prepared_opts)) prepare(G, o);
    ensure_pc(G, o.n_s);
    ensure_outer(G, o.restart);
    double t1 = now_ms();
    int B = (int)G->bodies.size();
    int nuo = B * (G->d + G->rot());
    for (int i = 0; i < nuo; ++i)
        if (!std::isfinite(body_UO[i])) throw Error{IBR_ENUMERIC, "body_UO contains NaN/Inf"};
    // prescribed bodies' velocities (free bodies' rows zeroed: their markers
    // have W = 0) and free bodies' loads
    std::vector<double> uo(body_UO, body_UO + nuo), load;
    int nr = G->d + G->rot();
    for (int bi = 0; bi < B; ++bi)
        if (G->bfree[bi] >= 0) {
            load.insert(load.end(), uo.begin() + bi * nr, uo.begin() + (bi + 1) * nr);
            std::fill(uo.begin() + bi * nr, uo.begin() + (bi + 1) * nr, 0.0);
        }
    IBR_CUDA_TRY(cudaMemcpyAsync(G->UO, uo.data(), nuo * sizeof(double), cudaMemcpyHostToDevice, s));
    // b = [g; 0; W = -K U; F]
    long long nS = G->nS;
    IBR_CUDA_TRY(cudaMemsetAsync(G->b, 0, nS * sizeof(double), s));
    if (gforce) {
        size_t bytes = (size_t)G->d * G->geo.ncell * sizeof(double);
        IBR_CUDA_TRY(cudaMemcpyAsync(G->b, gforce, bytes,
                                     g_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    }
    rigid_K(G->d, G->N, G->md.rel, G->md.body, G->UO, G->b + nS, -1.0, s);
    if (G->walls()) {
        // no net flux through the walls (solvability of the divergence rows)
        double flux = 0.0, scale = 0.0;
        for (int a = 0; a < G->d; ++a) {
            if (!((G->geo.wall >> a) & 1)) continue;
            const long long nf = G->face_points(a);
            const double* lo = G->wdata_host[2 * a].data() + (size_t)a * nf;
            const double* hi = G->wdata_host[2 * a + 1].data() + (size_t)a * nf;
            for (long long t = 0; t < nf; ++t) {
                flux += hi[t] - lo[t];
                scale += std::fabs(hi[t]) + std::fabs(lo[t]);
            }
        }
        require(std::fabs(flux) <= 1e-10 * scale, "the wall velocities have a net flux (inflow != outflow)");
        for (int a = 0; a < G->d; ++a)
            if ((G->geo.wall >> a) & 1)
                for (int sd = 0; sd < 2; ++sd) wall_lift(G->geo, a, sd, G->wdata[2 * a + sd], G->b, G->eta, s);
    }
    if (G->nfree > 0)
        IBR_CUDA_TRY(cudaMemcpyAsync(G->b + nS + (long long)G->N * G->d, load.data(),
                                     load.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    auto setup_pc = [&](auto* pc) {
        pc->ns = o.n_s;
        pc->pre = o.mg_pre;
        pc->post = o.mg_post;
        pc->variant = o.variant;
        pc->ps_count = 0;
    };
    if (G->precision == IBR_FP64) {
        setup_pc(G->pc64);
        G->pc64->Minv = G->Minv64;
        G->pc64->setup_free();
    } else {
        setup_pc(G->pc32);
        G->pc32->Minv = G->Minv32;
        G->pc32->setup_free();
    }
    int status = fgmres(G, o, info, warm);
    if (G->walls())
        for (int a = 0; a < G->d; ++a)
            if ((G->geo.wall >> a) & 1) wall_set_faces(G->geo, a, G->wdata[2 * a], G->x, s);
    IBR_CUDA_TRY(cudaStreamSynchronize(s));
    double t2 = now_ms();
    info.ms_setup = t1 - t0;
    info.ms_solve = t2 - t1;
    info.ps_applications =
        (int)(G->precision == IBR_FP64 ? G->pc64->ps_count : G->pc32->ps_count);
    G->have_solution = true;
    return status;
}

namespace ibr {

// Device bytes one grid holds through a solve with these sizes: the outer
// FGMRES workspace (double-float basis, Z, b, x, w), the preconditioner in its
// precision (multigrid levels, inner GMRES basis, P_S work), the marker data
// and gather lists of S, and the dense mobility blocks (as built, factorised,
// plus the factorisation's work block).  Every allocation of >= 1 MiB is
// rounded up to the 2 MiB page the CUDA allocator hands out; the many small
// buffers are covered by a fixed 16 MiB.  Periodic grids, prescribed bodies.
long long estimate_grid_bytes(int d, const int* n, int B, const int* Nb, int restart, int ns, int precision,
                              int mob_model) {
    auto pg = [](double b) {
        const double MiB = 1048576.0;
        return b >= MiB ? std::ceil(b / (2 * MiB)) * 2 * MiB : b;
    };
    const double e = precision == IBR_FP64 ? 8.0 : 4.0;
    Geo g = make_geo(d, n, 1.0);
    const double nc = (double)g.ncell;
    const double nS = (d + 1) * nc;
    long long N = 0;
    double blk2 = 0.0, blkmax = 0.0;
    for (int b = 0; b < B; ++b) {
        N += Nb[b];
        double m = (double)Nb[b] * d;
        blk2 += m * m;
        blkmax = std::max(blkmax, m * m);
    }
    const double dN = (double)N * d;
    const double len = nS + dN;
    const double lp = (double)(((long long)len + 1) & ~1LL);
    const int m = restart;
    double t = 0.0;
    // outer FGMRES
    t += pg(8.0 * (m + 1) * lp) + pg(8.0 * m * len) + 3 * pg(8.0 * len) + pg(8.0 * lp);
    t += 8.0 * ((m + 1) * (m + 1) + 8 * (m + 2)) + pg(8.0 * RED_BLOCKS * std::max(m + 1, 4));
    // preconditioner: coarse multigrid levels (d stacked fields, u and f)
    Geo c = g;
    while (Multigrid<float>::can_coarsen(c)) {
        c.n0 /= 2;
        c.n1 /= 2;
        if (d == 3) c.n2 /= 2;
        c.ncell = (long long)c.n0 * c.n1 * c.n2;
        t += 2 * pg(e * d * (double)c.ncell);
    }
    t += pg(e * (ns + 1) * nS) + pg(e * ns * nS) + 4 * pg(e * nS) + pg(e * d * nc) + 3 * pg(e * nc);
    t += pg(8.0 * RED_BLOCKS * std::max(ns + 1, 4)) + 2 * pg(e * dN) + pg(8.0 * dN);
    // the red-black split copies of u and f of the finest level and level 1 (periodic 3-D)
    if (d == 3 && g.n0 % 8 == 0) t += 2 * pg(e * d * nc);
    if (d == 3 && g.n0 % 16 == 0 && Multigrid<float>::can_coarsen(g)) t += 2 * pg(e * d * nc / 8);
    // markers: positions, lever arms, windows (index, FP64 and FP32 weights),
    // face-major gather lists (at most 4^d faces per marker and component)
    const double win = (double)N * d * d * 4;
    const double E = (double)N * d * std::pow(4.0, d);
    t += 2 * pg(8.0 * dN) + pg(4.0 * win) + pg(8.0 * win) + pg(4.0 * win);
    t += pg(8.0 * E) + pg(4.0 * E) + pg(4.0 * E) + pg(8.0 * E) + pg(4.0 * E);
    // the gather-list build's temporaries (sort keys, flags, positions)
    t += pg(8.0 * E) + 2 * pg(4.0 * E);
    // IBR_MOB_PAIR: the table (resident) and, while it is built, an FP64
    // preconditioner with PAIR_NS inner vectors and four solve vectors; its
    // blocks: one for all markers while d N <= PAIR_FULL_MAX
    if (mob_model == IBR_MOB_PAIR) {
        t += pg(4.0 * PAIR_S * d * d * nc);
        double mg64 = 0.0;
        Geo c2 = g;
        while (Multigrid<double>::can_coarsen(c2)) {
            c2.n0 /= 2;
            c2.n1 /= 2;
            if (d == 3) c2.n2 /= 2;
            c2.ncell = (long long)c2.n0 * c2.n1 * c2.n2;
            mg64 += 2 * pg(8.0 * d * (double)c2.ncell);
        }
        t += mg64 + pg(8.0 * (PAIR_NS + 1) * nS) + pg(8.0 * PAIR_NS * nS) + 8 * pg(8.0 * nS) + pg(8.0 * d * nc) +
             3 * pg(8.0 * nc);
        if (dN <= (double)pair_full_max()) blk2 = blkmax = dN * dN;
    }
    // coupled analytic forms within the single-block limit: one block of all markers
    if ((mob_model & IBR_MOB_COUPLED) && dN <= (double)pair_full_max()) blk2 = blkmax = dN * dN;
    // mobility: built (FP64) + factorised inverse (precision) + work: the FP64
    // path's work block, or the tensor-core path's two padded blocks
    t += pg(8.0 * blk2) + pg(e * blk2);
    if (precision == IBR_FP64) {
        t += pg(e * blkmax);
    } else {
        // padded block, X = L^-1, X^T, the recursion's product buffer (np^2 / 4),
        // the diagonal inverses, and the packed TF32 hi / lo operands of the
        // largest product
        const double np = std::ceil(std::sqrt(blkmax) / 128.0) * 128.0;
        t += 3 * pg(4.0 * np * np) + pg(np * np + 4.0 * 128.0 * 128.0) + pg(4.0 * np * 128.0) + pg(8.0 * np * np);
    }
    return (long long)(t + 16.0 * 1048576.0);
}

// a grid reused for another problem of the same shape: bodies dropped (the
// next solve rebins, rebuilds and refactorises), workspaces kept
void grid_clear_bodies(ibr_grid* G) {
    G->bodies.clear();
    G->dirty = true;
    G->have_solution = false;
}

// the stream the grid's work is issued on from now on (the grid must be idle)
void grid_set_stream(ibr_grid* G, cudaStream_t s) {
    if (G->own_stream) {
        cudaStreamDestroy(G->stream);
        G->own_stream = false;
    }
    G->stream = s;
}

}  // namespace ibr

// makes G->x usable as a state: set-up, workspaces, and x = 0 with the wall
// values on the wall faces if there is no solution yet
void ensure_state(ibr_grid* G, const ibr_solve_opts& o) {
    if (G->dirty || !mob_opts_equal(o, G->prepared_opts)) prepare(G, o);
    ensure_pc(G, o.n_s > 0 ? o.n_s : (G->walls() ? 4 : 2));
    ensure_outer(G, o.restart);
    if (!G->have_solution) {
        IBR_CUDA_TRY(cudaMemsetAsync(G->x, 0, G->len * sizeof(double), G->stream));
        for (int a = 0; a < G->d; ++a)
            if ((G->geo.wall >> a) & 1) wall_set_faces(G->geo, a, G->wdata[2 * a], G->x, G->stream);
        G->have_solution = true;
        G->adv_hist = false;
    }
    const long long m = (long long)G->d * G->geo.ncell;
    for (double** p : {&G->adv_v, &G->adv_N, &G->adv_Np, &G->adv_g})
        if (!*p) *p = dalloc<double>(m);
}

extern "C" {

const char* ibr_last_error(void) { return ibr::g_last_error.c_str(); }

int ibr_solve_opts_default(ibr_solve_opts* o) {
    if (!o) {
        ibr::set_error("ibr_solve_opts_default: NULL");
        return IBR_EINVAL;
    }
    opts_default(o);
    return IBR_OK;
}

int ibr_create_grid(ibr_grid** out, int dim, const int* n, const double* L, const int* bc, double eta, double rho,
                    double dt, int kernel, int precision, void* cuda_stream) {
    return run_guarded("ibr_create_grid", [&] {
        require(out != nullptr, "out is NULL");
        *out = nullptr;
        require(dim == 2 || dim == 3, "dim must be 2 or 3");
        require(n && L && bc, "n, L, bc must be non-NULL");
        int wall = 0;
        for (int a = 0; a < dim; ++a) {
            require(n[a] >= 4 && n[a] % 2 == 0, "each n[a] must be even and >= 4");
            require(L[a] > 0, "L[a] must be positive");
            auto is_wall = [](int b) { return b == IBR_NOSLIP || b == IBR_VELOCITY; };
            const bool per = bc[2 * a] == IBR_PERIODIC && bc[2 * a + 1] == IBR_PERIODIC;
            const bool wl = is_wall(bc[2 * a]) && is_wall(bc[2 * a + 1]);
            require(per || wl,
                    "each axis must be periodic at both ends or bounded by walls (IBR_NOSLIP / IBR_VELOCITY) at both "
                    "ends");
            if (wl) wall |= 1 << a;
        }
        double h = L[0] / n[0];
        for (int a = 1; a < dim; ++a)
            require(std::fabs(L[a] / n[a] - h) <= 1e-12 * h, "cells must be cubes (L[a]/n[a] equal)");
        require(eta > 0, "eta must be positive");
        require(rho >= 0 && dt >= 0, "rho, dt must be >= 0");
        require(kernel == IBR_KERNEL_PESKIN4 || kernel == IBR_KERNEL_BKP6,
                "kernel must be IBR_KERNEL_PESKIN4 or IBR_KERNEL_BKP6");
        require(kernel == IBR_KERNEL_PESKIN4 || wall == 0, "IBR_KERNEL_BKP6 needs a periodic box");
        require(precision == IBR_FP64 || precision == IBR_MIXED, "precision must be IBR_FP64 or IBR_MIXED");
        std::unique_ptr<ibr_grid> G(new ibr_grid());
        G->d = dim;
        for (int a = 0; a < dim; ++a) {
            G->n[a] = n[a];
            G->L[a] = L[a];
        }
        G->h = h;
        G->eta = eta;
        G->rho = rho;
        G->dt = dt;
        G->vol = 1.0;
        for (int a = 0; a < dim; ++a) G->vol *= L[a];
        G->precision = precision;
        G->geo = make_geo(dim, n, h);
        G->geo.wall = wall;
        G->geo.kw = kernel == IBR_KERNEL_BKP6 ? 6 : 4;
        require(G->geo.ncell < (1LL << 31), "a field must have fewer than 2^31 cells");
        G->nS = (long long)(dim + 1) * G->geo.ncell;
        G->len = G->nS;
        // the coarsest multigrid level must fit one CTA's shared memory
        {
            Geo g = G->geo;
            while (Multigrid<double>::can_coarsen(g)) {
                g.n0 /= 2;
                g.n1 /= 2;
                if (dim == 3) g.n2 /= 2;
                g.ncell = (long long)g.n0 * g.n1 * g.n2;
            }
            require(g.ncell <= 2048, "grid does not coarsen to <= 2048 cells (use sizes with more factors of 2)");
        }
        if (cuda_stream) {
            G->stream = (cudaStream_t)cuda_stream;
        } else {
            // a blocking stream: ordered with work on the legacy default stream
            IBR_CUDA_TRY(cudaStreamCreateWithFlags(&G->stream, cudaStreamDefault));
            G->own_stream = true;
        }
        // wall data, zero until ibr_set_boundary_velocity
        for (int a = 0; a < dim; ++a) {
            if (!((wall >> a) & 1)) continue;
            for (int sd = 0; sd < 2; ++sd) {
                const int f = 2 * a + sd;
                G->bc[f] = bc[f];
                const size_t cnt = (size_t)dim * G->face_points(a);
                G->wdata_host[f].assign(cnt, 0.0);
                G->wdata[f] = dalloc<double>(cnt);
                IBR_CUDA_TRY(cudaMemsetAsync(G->wdata[f], 0, cnt * sizeof(double), G->stream));
            }
        }
        opts_default(&G->prepared_opts);
        *out = G.release();
    });
}

int ibr_add_body(ibr_grid* G, const double* x_c, const double* quat, int kinematics, int* body_id) {
    return run_guarded("ibr_add_body", [&] {
        require(G && x_c, "grid and x_c must be non-NULL");
        require(kinematics == IBR_PRESCRIBED || kinematics == IBR_FREE, "kinematics must be IBR_PRESCRIBED or IBR_FREE");
        Body b;
        for (int a = 0; a < G->d; ++a) b.xc[a] = x_c[a];
        if (quat) quat_to_R(quat, b.R);
        b.kin = kinematics;
        G->bodies.push_back(b);
        if (body_id) *body_id = (int)G->bodies.size() - 1;
        G->dirty = true;
        G->have_solution = false;
    });
}

int ibr_set_markers(ibr_grid* G, int body_id, const double* r_body, int N) {
    return run_guarded("ibr_set_markers", [&] {
        require(G, "grid is NULL");
        require(body_id >= 0 && body_id < (int)G->bodies.size(), "bad body_id");
        require(N >= 1 && r_body, "N >= 1 and r_body non-NULL required");
        for (long long i = 0; i < (long long)N * G->d; ++i)
            if (!std::isfinite(r_body[i])) throw Error{IBR_ENUMERIC, "marker offsets contain NaN/Inf"};
        Body& b = G->bodies[body_id];
        b.rbody.assign(r_body, r_body + (size_t)N * G->d);
        b.N = N;
        G->dirty = true;
        G->have_solution = false;
    });
}

int ibr_set_boundary_velocity(ibr_grid* G, int face, const double* values) {
    return run_guarded("ibr_set_boundary_velocity", [&] {
        require(G != nullptr && values != nullptr, "grid and values must be non-NULL");
        require(face >= 0 && face < 2 * G->d, "face must be in [0, 2*dim)");
        require(G->bc[face] == IBR_VELOCITY, "face is not an IBR_VELOCITY wall");
        const size_t cnt = (size_t)G->d * G->face_points(face / 2);
        for (size_t i = 0; i < cnt; ++i)
            if (!std::isfinite(values[i])) throw Error{IBR_ENUMERIC, "boundary values contain NaN/Inf"};
        G->wdata_host[face].assign(values, values + cnt);
        IBR_CUDA_TRY(cudaMemcpyAsync(G->wdata[face], G->wdata_host[face].data(), cnt * sizeof(double),
                                     cudaMemcpyHostToDevice, G->stream));
        G->dirty = true;  // the marker check against walls with data runs in the set-up
        G->have_solution = false;
    });
}

int ibr_prepare(ibr_grid* G, const ibr_solve_opts* opts) {
    return run_guarded("ibr_prepare", [&] {
        require(G, "grid is NULL");
        ibr_solve_opts o;
        if (opts)
            o = *opts;
        else
            opts_default(&o);
        prepare(G, o);
    });
}

int ibr_solve_coupled(ibr_grid* G, const double* body_UO, const double* gforce, int g_on_device,
                      const ibr_solve_opts* opts, ibr_solve_info* info_out) {
    ibr_solve_info info;
    std::memset(&info, 0, sizeof(info));
    int status = IBR_OK;
    int rc = run_guarded("ibr_solve_coupled", [&] {
        require(G && body_UO, "grid and body_UO must be non-NULL");
        status = solve_core(G, body_UO, gforce, g_on_device, opts, info, false);
    });
    if (rc == IBR_OK && status != IBR_OK) {
        rc = status;
        ibr::set_error(status == IBR_ENOTCONV ? "ibr_solve_coupled: max_iters reached"
                                              : "ibr_solve_coupled: time cap reached");
    }
    info.status = rc;
    if (info_out) *info_out = info;
    return rc;
}

int ibr_set_velocity(ibr_grid* G, const double* v, int on_device) {
    return run_guarded("ibr_set_velocity", [&] {
        require(G && v, "grid and v must be non-NULL");
        ibr_solve_opts o = G->prepared_opts;
        ensure_state(G, o);
        cudaStream_t s = G->stream;
        const long long m = (long long)G->d * G->geo.ncell;
        IBR_CUDA_TRY(cudaMemsetAsync(G->x, 0, G->len * sizeof(double), s));
        IBR_CUDA_TRY(cudaMemcpyAsync(G->x, v, m * sizeof(double),
                                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        for (int a = 0; a < G->d; ++a)
            if ((G->geo.wall >> a) & 1) wall_set_faces(G->geo, a, G->wdata[2 * a], G->x, s);
        IBR_CUDA_TRY(cudaStreamSynchronize(s));
        G->have_solution = true;
        G->adv_hist = false;
    });
}

int ibr_advance(ibr_grid* G, const double* body_UO, const double* gforce, int g_on_device, int nsteps,
                double steady_tol, const ibr_solve_opts* opts, ibr_step_info* out) {
    ibr_step_info si;
    std::memset(&si, 0, sizeof(si));
    int status = IBR_OK;
    double t0 = now_ms();
    int rc = run_guarded("ibr_advance", [&] {
        require(G && body_UO, "grid and body_UO must be non-NULL");
        require(!G->steady(), "time stepping needs rho > 0 and dt > 0");
        require(nsteps >= 1, "nsteps must be >= 1");
        require(steady_tol >= 0.0, "steady_tol must be >= 0");
        ibr_solve_opts o;
        if (opts)
            o = *opts;
        else
            opts_default(&o);
        ensure_state(G, o);
        cudaStream_t s = G->stream;
        const Geo& g = G->geo;
        const long long m = (long long)G->d * g.ncell;
        if (gforce) {
            if (!G->adv_f) G->adv_f = dalloc<double>(m);
            IBR_CUDA_TRY(cudaMemcpyAsync(G->adv_f, gforce, m * sizeof(double),
                                         g_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        }
        WallData wd;
        for (int f = 0; f < 6; ++f) wd.data[f] = G->wdata[f];
        for (int step = 0; step < nsteps; ++step) {
            // g = (rho/dt) v^n - rho (3/2 N(v^n) - 1/2 N(v^{n-1})) (+ f); Euler on the first step
            IBR_CUDA_TRY(cudaMemcpyAsync(G->adv_v, G->x, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
            advect(g, G->adv_v, wd, G->adv_N, s);
            const bool ab2 = G->adv_hist;
            step_force(m, G->adv_v, G->adv_N, ab2 ? G->adv_Np : G->adv_N, gforce ? G->adv_f : nullptr, G->sigma(),
                       G->rho * (ab2 ? 1.5 : 1.0), G->rho * (ab2 ? -0.5 : 0.0), G->adv_g, s);
            ibr_solve_info info;
            std::memset(&info, 0, sizeof(info));
            status = solve_core(G, body_UO, G->adv_g, 1, &o, info, true);
            si.steps = step + 1;
            si.iters_total += info.iters;
            si.iters_last = info.iters;
            si.rel_res_last = info.rel_res_true;
            // ||v^{n+1} - v^n|| / ||v^{n+1}||
            IBR_CUDA_TRY(cudaMemcpyAsync(G->adv_g, G->x, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
            vec_axpby<double>(m, -1.0, G->adv_v, 1.0, G->adv_g, s);
            norm2<double>(m, G->adv_g, G->partial, G->sc + 4, s);
            norm2<double>(m, G->x, G->partial, G->sc + 5, s);
            IBR_CUDA_TRY(cudaMemcpyAsync(G->host_sc + 4, G->sc + 4, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
            IBR_CUDA_TRY(cudaStreamSynchronize(s));
            const double num = std::sqrt(G->host_sc[4]), den = std::sqrt(G->host_sc[5]);
            si.change = den > 0.0 ? num / den : 0.0;
            std::swap(G->adv_N, G->adv_Np);
            G->adv_hist = true;
            if (status != IBR_OK) break;
            if (si.change <= steady_tol) break;
        }
    });
    if (rc == IBR_OK && status != IBR_OK) {
        rc = status;
        ibr::set_error(status == IBR_ENOTCONV ? "ibr_advance: a step's solve reached max_iters"
                                              : "ibr_advance: a step's solve reached the time cap");
    }
    si.status = rc;
    si.ms = now_ms() - t0;
    if (out) *out = si;
    return rc;
}

int ibr_op_advect(ibr_grid* G, const double* v, double* N) {
    return run_guarded("ibr_op_advect", [&] {
        require(G && v && N, "grid, v, N must be non-NULL");
        WallData wd;
        for (int f = 0; f < 6; ++f) wd.data[f] = G->wdata[f];
        advect(G->geo, v, wd, N, G->stream);
    });
}

int ibr_get_forces(ibr_grid* G, double* Lambda, double* body_FT) {
    return run_guarded("ibr_get_forces", [&] {
        require(G, "grid is NULL");
        if (!G->have_solution) throw Error{IBR_ESTATE, "no solution (call ibr_solve_coupled first)"};
        cudaStream_t s = G->stream;
        const double* lam = G->x + G->nS;
        if (Lambda)
            IBR_CUDA_TRY(cudaMemcpyAsync(Lambda, lam, sizeof(double) * G->N * G->d, cudaMemcpyDeviceToHost, s));
        if (body_FT) {
            rigid_KT(G->d, (int)G->bodies.size(), G->md.body_start, G->md.rel, lam, G->FT, s);
            IBR_CUDA_TRY(cudaMemcpyAsync(body_FT, G->FT, sizeof(double) * G->bodies.size() * (G->d + G->rot()),
                                         cudaMemcpyDeviceToHost, s));
        }
        IBR_CUDA_TRY(cudaStreamSynchronize(s));
    });
}

int ibr_get_body_velocities(ibr_grid* G, const double* body_UO, double* out) {
    return run_guarded("ibr_get_body_velocities", [&] {
        require(G && body_UO && out, "grid, body_UO, out must be non-NULL");
        if (!G->have_solution) throw Error{IBR_ESTATE, "no solution (call ibr_solve_coupled first)"};
        int B = (int)G->bodies.size(), nr = G->d + G->rot();
        std::copy(body_UO, body_UO + (size_t)B * nr, out);
        if (G->nfree > 0) {
            std::vector<double> U(G->nU);
            IBR_CUDA_TRY(cudaMemcpyAsync(U.data(), G->x + G->nS + (long long)G->N * G->d, G->nU * sizeof(double),
                                         cudaMemcpyDeviceToHost, G->stream));
            IBR_CUDA_TRY(cudaStreamSynchronize(G->stream));
            for (int bi = 0; bi < B; ++bi)
                if (G->bfree[bi] >= 0) std::copy(U.begin() + G->bfree[bi] * nr, U.begin() + (G->bfree[bi] + 1) * nr,
                                                 out + (size_t)bi * nr);
        }
    });
}

int ibr_get_fields(ibr_grid* G, double* v, double* p, int to_device) {
    return run_guarded("ibr_get_fields", [&] {
        require(G, "grid is NULL");
        if (!G->have_solution) throw Error{IBR_ESTATE, "no solution (call ibr_solve_coupled first)"};
        cudaStream_t s = G->stream;
        long long n = G->geo.ncell;
        cudaMemcpyKind kind = to_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (v) IBR_CUDA_TRY(cudaMemcpyAsync(v, G->x, sizeof(double) * G->d * n, kind, s));
        if (p) IBR_CUDA_TRY(cudaMemcpyAsync(p, G->x + (long long)G->d * n, sizeof(double) * n, kind, s));
        IBR_CUDA_TRY(cudaStreamSynchronize(s));
    });
}

int ibr_sizes(const ibr_grid* G, long long* system_len, int* n_markers, int* n_bodies) {
    return run_guarded("ibr_sizes", [&] {
        require(G, "grid is NULL");
        int N = 0;
        for (auto& b : G->bodies) N += b.N;
        int nfree = 0;
        for (auto& b : G->bodies) nfree += b.kin == IBR_FREE;
        if (system_len) *system_len = G->nS + (long long)N * G->d + (long long)nfree * (G->d + G->rot());
        if (n_markers) *n_markers = N;
        if (n_bodies) *n_bodies = (int)G->bodies.size();
    });
}

static void need_prepared(ibr_grid* G) {
    require(G != nullptr, "grid is NULL");
    if (G->dirty) throw Error{IBR_ESTATE, "geometry changed: call ibr_prepare or ibr_solve_coupled first"};
}

int ibr_apply_system(ibr_grid* G, const double* x, double* y) {
    return run_guarded("ibr_apply_system", [&] {
        need_prepared(G);
        require(x && y, "x, y must be non-NULL");
        if (!G->shift) G->shift = dalloc<double>(4);
        full_matvec(G, x, y);
    });
}

int ibr_op_spread(ibr_grid* G, const double* lam, double* f) {
    return run_guarded("ibr_op_spread", [&] {
        need_prepared(G);
        require(lam && f, "lam, f must be non-NULL");
        cudaStream_t s = G->stream;
        long long n = G->geo.ncell;
        IBR_CUDA_TRY(cudaMemsetAsync(f, 0, sizeof(double) * G->d * n, s));
        spread_gather<double>(G->md, lam, f, 1.0 / std::pow(G->h, G->d), s);
        if (G->null_v()) {
            if (!G->shift) G->shift = dalloc<double>(4);
            lam_sum<double>(G->d, G->N, lam, 1.0 / G->vol, G->shift, s);
            subtract_means<double>(n, G->d, f, G->shift, s);
        }
    });
}

int ibr_op_interp(ibr_grid* G, const double* v, double* U) {
    return run_guarded("ibr_op_interp", [&] {
        need_prepared(G);
        require(v && U, "v, U must be non-NULL");
        interp<double, double>(G->geo, G->md, v, U, 1.0, nullptr, G->stream, 0.0);
    });
}

int ibr_op_rigid(ibr_grid* G, const double* UO, double* V) {
    return run_guarded("ibr_op_rigid", [&] {
        need_prepared(G);
        require(UO && V, "UO, V must be non-NULL");
        rigid_K(G->d, G->N, G->md.rel, G->md.body, UO, V, 1.0, G->stream);
    });
}

int ibr_op_rigid_T(ibr_grid* G, const double* lam, double* FT) {
    return run_guarded("ibr_op_rigid_T", [&] {
        need_prepared(G);
        require(lam && FT, "lam, FT must be non-NULL");
        rigid_KT(G->d, (int)G->bodies.size(), G->md.body_start, G->md.rel, lam, FT, G->stream);
    });
}

int ibr_op_mtilde(ibr_grid* G, int body, double* out) {
    return run_guarded("ibr_op_mtilde", [&] {
        need_prepared(G);
        require(body >= 0 && body < G->nblk, "bad mobility block");
        require(out, "out must be non-NULL");
        long long cnt = G->moff[body + 1] - G->moff[body];
        IBR_CUDA_TRY(cudaMemcpyAsync(out, G->Mbuild + G->moff[body], cnt * sizeof(double), cudaMemcpyDeviceToDevice,
                                     G->stream));
    });
}

int ibr_op_mtilde_solve(ibr_grid* G, const double* rhs, double* out) {
    return run_guarded("ibr_op_mtilde_solve", [&] {
        need_prepared(G);
        require(rhs && out, "rhs, out must be non-NULL");
        cudaStream_t s = G->stream;
        int dN = G->N * G->d;
        if (G->precision == IBR_FP64) {
            blockdiag_gemv<double, double>(G->nblk, G->moff_dev, G->roff_dev, dN, G->Minv64, rhs, out, s);
        } else {
            ensure_pc(G, std::max(G->pc_ns, 1));
            float* tin = G->pc32->dU;
            float* tout = G->pc32->lamT;
            vec_convert<double, float>(dN, rhs, tin, s);
            blockdiag_gemv<float, float>(G->nblk, G->moff_dev, G->roff_dev, dN, G->Minv32, tin, tout, s);
            vec_convert<float, double>(dN, tout, out, s);
        }
    });
}

int ibr_op_stokes_pc(ibr_grid* G, const double* r, double* z) {
    return run_guarded("ibr_op_stokes_pc", [&] {
        require(G && r && z, "grid, r, z must be non-NULL");
        cudaStream_t s = G->stream;
        long long nS = G->nS;
        ensure_pc(G, std::max(G->pc_ns, 1));
        if (G->precision == IBR_FP64) {
            G->pc64->apply_ps(r, z);
        } else {
            vec_convert<double, float>(nS, r, G->pc32->rs, s);
            G->pc32->apply_ps(G->pc32->rs, G->pc32->xs);
            vec_convert<float, double>(nS, G->pc32->xs, z, s);
        }
    });
}

int ibr_op_vcycle(ibr_grid* G, double sigma, double kappa, const double* f, double* u, int k) {
    return run_guarded("ibr_op_vcycle", [&] {
        require(G && f && u, "grid, f, u must be non-NULL");
        require(k >= 1 && sigma >= 0 && kappa > 0, "k >= 1, sigma >= 0, kappa > 0 required");
        cudaStream_t s = G->stream;
        long long n = G->geo.ncell;
        ensure_pc(G, std::max(G->pc_ns, 1));
        if (G->precision == IBR_FP64) {
            auto* pc = G->pc64;
            for (int i = 0; i < k; ++i) pc->mg.vcycle(u, f, 1, FLD_P, sigma, kappa, false, pc->pre, pc->post, s);
        } else {
            auto* pc = G->pc32;
            vec_convert<double, float>(n, f, pc->rs, s);
            vec_convert<double, float>(n, u, pc->xs, s);
            for (int i = 0; i < k; ++i) pc->mg.vcycle(pc->xs, pc->rs, 1, FLD_P, sigma, kappa, false, pc->pre, pc->post, s);
            vec_convert<float, double>(n, pc->xs, u, s);
        }
    });
}

int ibr_op_gemm_tf32x3(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                       float alpha, float beta, void* cuda_stream) {
    return run_guarded("ibr_op_gemm_tf32x3", [&] {
        require(A && B && C, "A, B, C must be non-NULL");
        require(M >= 0 && N >= 0 && K >= 0 && lda >= K && ldb >= K && ldc >= N, "bad sizes");
        cudaStream_t s = (cudaStream_t)cuda_stream;
        int* err = nullptr;
        IBR_CUDA_TRY(cudaMallocAsync(&err, sizeof(int), s));
        IBR_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
        int herr = 0;
        try {
            gemm_tf32x3(M, N, K, A, lda, B, ldb, C, ldc, alpha, beta, false, err, s);
            IBR_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
            IBR_CUDA_TRY(cudaStreamSynchronize(s));
        } catch (...) {
            cudaFreeAsync(err, s);
            throw;
        }
        IBR_CUDA_TRY(cudaFreeAsync(err, s));
        if (herr) throw Error{IBR_ECUDA, "a tensor-core product timed out waiting for its MMAs"};
    });
}

int ibr_mobility_defaults(int dim, int kernel, double* a_over_h, double* coef9) {
    return run_guarded("ibr_mobility_defaults", [&] {
        require(dim == 2 || dim == 3, "dim must be 2 or 3");
        require(kernel == IBR_KERNEL_PESKIN4 || kernel == IBR_KERNEL_BKP6, "unknown kernel");
        const bool six = kernel == IBR_KERNEL_BKP6;
        if (a_over_h) *a_over_h = dim == 3 ? (six ? 1.47 : 1.25) : (six ? AOH_2D_BKP6 : AOH_2D_PESKIN4);
        if (coef9)
            for (int q = 0; q < 9; ++q) coef9[q] = dim == 2 ? (six ? COEF_2D_BKP6 : COEF_2D_PESKIN4)[q] : 0.0;
    });
}

int ibr_tuned_vcycle_schedule(int idx, int* shape_l_c_esz, int* cluster_level) {
    return run_guarded("ibr_tuned_vcycle_schedule", [&] {
        int v[7];
        require(tuned_cluster(idx, v), "no tuned V-cycle schedule with this index");
        if (shape_l_c_esz)
            for (int q = 0; q < 6; ++q) shape_l_c_esz[q] = v[q];
        if (cluster_level) *cluster_level = v[6];
    });
}

int ibr_tuned_smoother_tile(int idx, int* shape_c_esz, int* by, int* kz) {
    return run_guarded("ibr_tuned_smoother_tile", [&] {
        int v[7];
        require(tuned_tile(idx, v), "no tuned tile with this index");
        if (shape_c_esz)
            for (int q = 0; q < 5; ++q) shape_c_esz[q] = v[q];
        if (by) *by = v[5];
        if (kz) *kz = v[6];
    });
}

int ibr_estimate_device_bytes(int dim, const int* n, int n_bodies, const int* n_markers, int restart, int n_s,
                              int precision, int mob_model, long long* bytes) {
    return run_guarded("ibr_estimate_device_bytes", [&] {
        require(bytes && n && (n_bodies == 0 || n_markers), "n, bytes (and n_markers) must be non-NULL");
        require(dim == 2 || dim == 3, "dim must be 2 or 3");
        require(n_bodies >= 0 && restart >= 1 && n_s >= 0, "n_bodies >= 0, restart >= 1, n_s >= 0 required");
        require(precision == IBR_FP64 || precision == IBR_MIXED, "bad precision");
        for (int a = 0; a < dim; ++a) require(n[a] >= 4, "n[a] >= 4 required");
        for (int b = 0; b < n_bodies; ++b) require(n_markers[b] >= 0, "n_markers must be >= 0");
        *bytes = estimate_grid_bytes(dim, n, n_bodies, n_markers, restart, n_s == 0 ? 2 : n_s, precision, mob_model);
    });
}

int ibr_destroy_grid(ibr_grid* G) {
    if (!G) return IBR_OK;
    return run_guarded("ibr_destroy_grid", [&] {
        cudaStreamSynchronize(G->stream);
        delete G->pc64;
        delete G->pc32;
        free_markers(G);
        free_outer(G);
        dfree(G->info_dev);
        if (G->host_sc) cudaFreeHost(G->host_sc);
        for (double* p : G->wdata) dfree(p);
        for (double** p : {&G->adv_v, &G->adv_N, &G->adv_Np, &G->adv_g, &G->adv_f}) dfree(*p);
        G->pair_hold.reset();  // the shared table goes with its last grid
        if (G->own_stream) cudaStreamDestroy(G->stream);
        delete G;
    });
}

}  // extern "C"
