// MAC-grid operators and the geometric multigrid pieces of P_S (Sec. V.B).
//
// Layout: a scalar field is ncell values, x fastest; a stack of C fields is
// C*ncell values.  A Stokes vector is [v_0 .. v_{d-1} | p].  All grids here
// are periodic with an even number of cells per axis (red-black ordering).
#include <cstdlib>
#include <cstring>

#include "ibr_internal.cuh"

namespace ibr {
namespace {

struct Nbr {
    long long c;          // flat index
    long long xp, xm;     // offsets to i+1, i-1 (wrapped)
    long long yp, ym;
    long long zp, zm;
};

template <int D>
__device__ __forceinline__ Nbr neighbours(const Geo& g, int i, int j, int k) {
    Nbr n;
    long long sy = g.n0;
    long long sz = (long long)g.n0 * g.n1;
    n.c = i + sy * j + sz * k;
    n.xp = (i == g.n0 - 1) ? -(long long)(g.n0 - 1) : 1;
    n.xm = (i == 0) ? (long long)(g.n0 - 1) : -1;
    n.yp = (j == g.n1 - 1) ? -(long long)(g.n1 - 1) * sy : sy;
    n.ym = (j == 0) ? (long long)(g.n1 - 1) * sy : -sy;
    if (D == 3) {
        n.zp = (k == g.n2 - 1) ? -(long long)(g.n2 - 1) * sz : sz;
        n.zm = (k == 0) ? (long long)(g.n2 - 1) * sz : -sz;
    } else {
        n.zp = n.zm = 0;
    }
    return n;
}

template <int D, typename T>
__device__ __forceinline__ T nbr_sum(const T* __restrict__ u, const Nbr& n) {
    T s = u[n.c + n.xp] + u[n.c + n.xm] + u[n.c + n.yp] + u[n.c + n.ym];
    if (D == 3) s += u[n.c + n.zp] + u[n.c + n.zm];
    return s;
}

// y_v^a = sigma v^a - kh2 (nbrsum - 2D v^a) + (p_c - p_{c-e_a}) ih + shift_a ;
// y_p = -ih sum_a (v^a_{c+e_a} - v^a_c)
template <int D, typename T>
__global__ void __launch_bounds__(256) k_stokes(const T* __restrict__ x, T* __restrict__ y, Geo g, T sigma, T kh2,
                                                T ih, const double* __restrict__ shift) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= g.ncell) return;
    int i = (int)(t % g.n0);
    long long r = t / g.n0;
    int j = (int)(r % g.n1);
    int k = (int)(r / g.n1);
    Nbr n = neighbours<D>(g, i, j, k);
    const T* p = x + D * g.ncell;
    T pc = p[n.c];
    T div = T(0);
    const long long pm[3] = {n.xm, n.ym, n.zm};
    const long long pp[3] = {n.xp, n.yp, n.zp};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const T* u = x + a * g.ncell;
        T uc = u[n.c];
        T lap = nbr_sum<D, T>(u, n) - T(2 * D) * uc;
        T val = sigma * uc - kh2 * lap + (pc - p[n.c + pm[a]]) * ih;
        if (shift) val += (T)shift[a];
        y[a * g.ncell + n.c] = val;
        div += u[n.c + pp[a]] - uc;
    }
    y[D * g.ncell + n.c] = -div * ih;
}

// red-black Gauss-Seidel half sweep on C stacked fields (component = blockIdx.y)
template <int D, typename T>
__global__ void __launch_bounds__(256) k_rbgs(T* __restrict__ u, const T* __restrict__ f, Geo g, T sigma, T kh2,
                                              int color, int zero_init) {
    long long half = g.ncell >> 1;
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= half) return;
    int cmp = blockIdx.y;
    T* uu = u + cmp * g.ncell;
    const T* ff = f + cmp * g.ncell;
    int hn0 = g.n0 >> 1;
    int ih = (int)(t % hn0);
    long long r = t / hn0;
    int j = (int)(r % g.n1);
    int k = (int)(r / g.n1);
    int i = 2 * ih + ((j + k + color) & 1);
    Nbr n = neighbours<D>(g, i, j, k);
    T nb = zero_init ? T(0) : nbr_sum<D, T>(uu, n);
    T diag = sigma + T(2 * D) * kh2;
    uu[n.c] = (ff[n.c] + kh2 * nb) / diag;
}

// One full red-black Gauss-Seidel sweep (colour c0 first, then 1 - c0) of a
// 3-D periodic field, out of place: u_new = sweep(u_old).  Same arithmetic and
// summation order as two k_rbgs half sweeps, so the result is identical.
// A CTA owns a FX x FY column of cells and marches along z over [z0, z0+FZ):
// at plane p it loads u_old(p+1) with a 2-cell in-plane halo, updates the
// first colour on plane p over the tile plus a 1-cell ring (recomputed by the
// neighbouring CTAs too, so no CTA reads another's output), then updates the
// second colour on plane p-1 from the first-colour values of planes p-2..p.
constexpr int FX = 32, FY = 8, FZ = 8;

template <typename T>
__global__ void __launch_bounds__(FX* FY) k_rbgs_fused3d(const T* __restrict__ uo, const T* __restrict__ f,
                                                         T* __restrict__ un, Geo g, T sigma, T kh2, int c0,
                                                         int zero_init) {
    __shared__ T su[3][FY + 4][FX + 4];   // u_old planes p-1, p, p+1 (ring)
    __shared__ T sr[3][FY + 2][FX + 2];   // first-colour values, planes p-2, p-1, p (ring)
    __shared__ T sf[2][FY + 2][FX + 2];   // f planes p-1, p (ring)
    const int cmp = blockIdx.z;
    const long long off = (long long)cmp * g.ncell;
    uo += off;
    f += off;
    un += off;
    const int ntx = g.n0 / FX;
    const int bx = (blockIdx.x % ntx) * FX, by = (blockIdx.x / ntx) * FY;
    const int z0 = blockIdx.y * FZ;
    const int z1 = min(z0 + FZ, g.n2);
    const int tid = threadIdx.x;
    const long long sy = g.n0, sz = (long long)g.n0 * g.n1;
    const T diag = sigma + T(6) * kh2;
    auto wrap = [](int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); };
    auto load_u = [&](int p) {
        int slot = ((p % 3) + 3) % 3, pz = wrap(p, g.n2);
        for (int e = tid; e < (FY + 4) * (FX + 4); e += FX * FY) {
            int ly = e / (FX + 4), lx = e % (FX + 4);
            int gx = wrap(bx + lx - 2, g.n0), gy = wrap(by + ly - 2, g.n1);
            su[slot][ly][lx] = zero_init ? T(0) : uo[gx + sy * gy + sz * pz];
        }
    };
    auto load_f = [&](int p) {
        int slot = ((p % 2) + 2) % 2, pz = wrap(p, g.n2);
        for (int e = tid; e < (FY + 2) * (FX + 2); e += FX * FY) {
            int ly = e / (FX + 2), lx = e % (FX + 2);
            int gx = wrap(bx + lx - 1, g.n0), gy = wrap(by + ly - 1, g.n1);
            sf[slot][ly][lx] = f[gx + sy * gy + sz * pz];
        }
    };
    load_u(z0 - 2);
    load_u(z0 - 1);
    for (int p = z0 - 1; p <= z1; ++p) {
        load_u(p + 1);
        load_f(p);
        __syncthreads();
        // first colour on plane p, tile + 1-cell ring
        {
            const int s0 = ((p - 1) % 3 + 3) % 3, s1 = ((p % 3) + 3) % 3, s2 = ((p + 1) % 3 + 3) % 3;
            const int fs = ((p % 2) + 2) % 2, rs = s1;
            for (int e = tid; e < (FY + 2) * (FX + 2); e += FX * FY) {
                int ly = e / (FX + 2), lx = e % (FX + 2);
                int gx = bx + lx - 1, gy = by + ly - 1;
                int pz = wrap(p, g.n2);
                int colour = (wrap(gx, g.n0) + wrap(gy, g.n1) + pz) & 1;
                if (colour != c0) continue;
                int ux = lx + 1, uy = ly + 1;
                // the association of nbr_sum: (x+ + x- + y+ + y-) + (z+ + z-)
                T nb = zero_init ? T(0)
                                 : (su[s1][uy][ux + 1] + su[s1][uy][ux - 1] + su[s1][uy + 1][ux] + su[s1][uy - 1][ux]) +
                                       (su[s2][uy][ux] + su[s0][uy][ux]);
                sr[rs][ly][lx] = (sf[fs][ly][lx] + kh2 * nb) / diag;
            }
        }
        __syncthreads();
        // second colour on plane p-1, tile interior; write both colours
        const int q = p - 1;
        if (q >= z0) {
            const int r0 = ((q - 1) % 3 + 3) % 3, r1 = ((q % 3) + 3) % 3, r2 = ((q + 1) % 3 + 3) % 3;
            const int fs = ((q % 2) + 2) % 2;
            int lx = tid % FX, ly = tid / FX;
            int gx = bx + lx, gy = by + ly, qz = wrap(q, g.n2);
            int colour = (gx + gy + qz) & 1;
            T val;
            if (colour == c0) {
                val = sr[r1][ly + 1][lx + 1];
            } else {
                T nb = (sr[r1][ly + 1][lx + 2] + sr[r1][ly + 1][lx] + sr[r1][ly + 2][lx + 1] + sr[r1][ly][lx + 1]) +
                       (sr[r2][ly + 1][lx + 1] + sr[r0][ly + 1][lx + 1]);
                val = (sf[fs][ly + 1][lx + 1] + kh2 * nb) / diag;
            }
            un[gx + sy * gy + sz * qz] = val;
        }
        __syncthreads();
    }
}

// coarse f = average over the 2^D children of the fine residual f - (sigma u - kh2 Lap u)
template <int D, typename T>
__global__ void __launch_bounds__(256) k_resid_restrict(const T* __restrict__ u, const T* __restrict__ f,
                                                        T* __restrict__ fc, Geo gf, Geo gc, T sigma, T kh2) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= gc.ncell) return;
    int cmp = blockIdx.y;
    const T* uu = u + cmp * gf.ncell;
    const T* ff = f + cmp * gf.ncell;
    int I = (int)(t % gc.n0);
    long long r = t / gc.n0;
    int J = (int)(r % gc.n1);
    int K = (int)(r / gc.n1);
    T acc = T(0);
#pragma unroll
    for (int c = 0; c < (1 << D); ++c) {
        int i = 2 * I + (c & 1);
        int j = 2 * J + ((c >> 1) & 1);
        int k = D == 3 ? 2 * K + ((c >> 2) & 1) : 0;
        Nbr n = neighbours<D>(gf, i, j, k);
        T uc = uu[n.c];
        T res = ff[n.c] - (sigma * uc - kh2 * (nbr_sum<D, T>(uu, n) - T(2 * D) * uc));
        acc += res;
    }
    fc[cmp * gc.ncell + t] = acc * (T(1) / T(1 << D));
}

// cell-centred (bi/tri)linear prolongation: weights 3/4 (parent), 1/4 (the
// neighbour on the side of the child) per axis; u += P uc
template <int D, typename T>
__global__ void __launch_bounds__(256) k_prolong(T* __restrict__ u, const T* __restrict__ uc, Geo gf, Geo gc) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= gf.ncell) return;
    int cmp = blockIdx.y;
    const T* cc = uc + cmp * gc.ncell;
    int i = (int)(t % gf.n0);
    long long r = t / gf.n0;
    int j = (int)(r % gf.n1);
    int k = (int)(r / gf.n1);
    int I[2], Jc[2], Kc[2];
    I[0] = i >> 1;
    I[1] = (i & 1) ? (I[0] + 1 == gc.n0 ? 0 : I[0] + 1) : (I[0] == 0 ? gc.n0 - 1 : I[0] - 1);
    Jc[0] = j >> 1;
    Jc[1] = (j & 1) ? (Jc[0] + 1 == gc.n1 ? 0 : Jc[0] + 1) : (Jc[0] == 0 ? gc.n1 - 1 : Jc[0] - 1);
    if (D == 3) {
        Kc[0] = k >> 1;
        Kc[1] = (k & 1) ? (Kc[0] + 1 == gc.n2 ? 0 : Kc[0] + 1) : (Kc[0] == 0 ? gc.n2 - 1 : Kc[0] - 1);
    } else {
        Kc[0] = Kc[1] = 0;
    }
    const T w[2] = {T(0.75), T(0.25)};
    T acc = T(0);
#pragma unroll
    for (int c = 0; c < (1 << D); ++c) {
        int a = c & 1, b = (c >> 1) & 1, e = D == 3 ? (c >> 2) & 1 : 0;
        T ww = w[a] * w[b] * (D == 3 ? w[e] : T(1));
        long long idx = I[a] + (long long)gc.n0 * (Jc[b] + (long long)gc.n1 * Kc[e]);
        acc += ww * cc[idx];
    }
    u[cmp * gf.ncell + t] += acc;
}

// single-CTA coarse solve: zero start, (mean-removed f if sigma == 0), red-black
// sweeps in shared memory, mean-removed result if sigma == 0.  One CTA per field.
template <int D, typename T>
__global__ void __launch_bounds__(1024) k_coarse(T* __restrict__ u, const T* __restrict__ f, Geo g, T sigma, T kh2,
                                                 int sweeps) {
    extern __shared__ unsigned char smem_raw[];
    T* su = reinterpret_cast<T*>(smem_raw);
    T* sf = su + g.ncell;
    __shared__ double red[32];
    int cmp = blockIdx.x;
    const T* ff = f + cmp * g.ncell;
    T* uu = u + cmp * g.ncell;
    int tid = threadIdx.x;
    int nt = blockDim.x;
    // mean of f
    double part = 0.0;
    for (long long c = tid; c < g.ncell; c += nt) {
        T v = ff[c];
        sf[c] = v;
        su[c] = T(0);
        part += (double)v;
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((tid & 31) == 0) red[tid >> 5] = part;
    __syncthreads();
    if (tid < 32) {
        double v = tid < (nt >> 5) ? red[tid] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (tid == 0) red[0] = v;
    }
    __syncthreads();
    T fmean = sigma == T(0) ? (T)(red[0] / (double)g.ncell) : T(0);
    __syncthreads();
    for (long long c = tid; c < g.ncell; c += nt) sf[c] -= fmean;
    __syncthreads();
    T diag = sigma + T(2 * D) * kh2;
    for (int s = 0; s < sweeps; ++s) {
        for (int color = 0; color < 2; ++color) {
            for (long long c = tid; c < g.ncell; c += nt) {
                int i = (int)(c % g.n0);
                long long r = c / g.n0;
                int j = (int)(r % g.n1);
                int k = (int)(r / g.n1);
                if (((i + j + k) & 1) != color) continue;
                Nbr n = neighbours<D>(g, i, j, k);
                su[c] = (sf[c] + kh2 * nbr_sum<D, T>(su, n)) / diag;
            }
            __syncthreads();
        }
    }
    part = 0.0;
    for (long long c = tid; c < g.ncell; c += nt) part += (double)su[c];
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = part;
    __syncthreads();
    if (tid < 32) {
        double v = tid < (nt >> 5) ? red[tid] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (tid == 0) red[0] = v;
    }
    __syncthreads();
    T umean = sigma == T(0) ? (T)(red[0] / (double)g.ncell) : T(0);
    for (long long c = tid; c < g.ncell; c += nt) uu[c] = su[c] - umean;
}

// q = -D y - hd ; qr = rhs_scale * q
template <int D, typename T>
__global__ void __launch_bounds__(256) k_ps_div(const T* __restrict__ y, const T* __restrict__ hd,
                                                T* __restrict__ qr, T rhs_scale, T* __restrict__ q, Geo g, T ih) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= g.ncell) return;
    int i = (int)(t % g.n0);
    long long r = t / g.n0;
    int j = (int)(r % g.n1);
    int k = (int)(r / g.n1);
    Nbr n = neighbours<D>(g, i, j, k);
    const long long pp[3] = {n.xp, n.yp, n.zp};
    T div = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const T* u = y + a * g.ncell;
        div += u[n.c + pp[a]] - u[n.c];
    }
    T qq = -div * ih - hd[n.c];
    q[n.c] = qq;
    qr[n.c] = rhs_scale * qq;
}

// z_v^a = y^a + h^2 (G phi)^a = y^a + h (phi_c - phi_{c-e_a}) ; z_p = c_q q + c_phi phi
template <int D, typename T>
__global__ void __launch_bounds__(256) k_ps_finish(const T* __restrict__ y, const T* __restrict__ phi,
                                                   const T* __restrict__ q, T* __restrict__ z, Geo g, T h, T c_q,
                                                   T c_phi) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= g.ncell) return;
    int i = (int)(t % g.n0);
    long long r = t / g.n0;
    int j = (int)(r % g.n1);
    int k = (int)(r / g.n1);
    Nbr n = neighbours<D>(g, i, j, k);
    const long long pm[3] = {n.xm, n.ym, n.zm};
    T pc = phi[n.c];
#pragma unroll
    for (int a = 0; a < D; ++a) z[a * g.ncell + n.c] = y[a * g.ncell + n.c] + h * (pc - phi[n.c + pm[a]]);
    z[D * g.ncell + n.c] = c_q * q[n.c] + c_phi * pc;
}

}  // namespace

template <typename T>
void stokes_apply(const Geo& g, const T* x, T* y, double sigma, double eta, const double* shift_dev,
                  cudaStream_t s) {
    T kh2 = (T)(eta / (g.h * g.h));
    T ih = (T)(1.0 / g.h);
    int nb = grid_1d(g.ncell, 256);
    ProfScope ps(KID_STOKES, s, 2.0 * (g.d + 1) * g.ncell * sizeof(T));
    if (g.d == 3)
        k_stokes<3, T><<<nb, 256, 0, s>>>(x, y, g, (T)sigma, kh2, ih, shift_dev);
    else
        k_stokes<2, T><<<nb, 256, 0, s>>>(x, y, g, (T)sigma, kh2, ih, shift_dev);
    IBR_CHECK_LAUNCH();
}

template <typename T>
void mg_smooth(const Geo& g, T* u, const T* f, int C, double sigma, double kappa, int color, bool zero_init,
               cudaStream_t s) {
    T kh2 = (T)(kappa / (g.h * g.h));
    dim3 grid(grid_1d(g.ncell / 2, 256), C);
    // half sweep: read the other colour and f of this colour, write this colour
    ProfScope ps(KID_RBGS, s, (zero_init ? 1.0 : 1.5) * C * g.ncell * sizeof(T));
    if (g.d == 3)
        k_rbgs<3, T><<<grid, 256, 0, s>>>(u, f, g, (T)sigma, kh2, color, zero_init ? 1 : 0);
    else
        k_rbgs<2, T><<<grid, 256, 0, s>>>(u, f, g, (T)sigma, kh2, color, zero_init ? 1 : 0);
    IBR_CHECK_LAUNCH();
}

// The fused sweep pays a serial z-march per CTA, so it is used only on levels
// large enough to fill the GPU (>= IBR_FUSED_MIN_CELLS cells, default 64^3);
// IBR_SMOOTHER=halfsweep selects the two-launch sweep everywhere (the two give
// identical results).
bool mg_fused_ok(const Geo& g) {
    static const long long min_cells = [] {
        const char* e = std::getenv("IBR_FUSED_MIN_CELLS");
        return e ? std::atoll(e) : 64LL * 64 * 64;
    }();
    static const bool off = [] {
        const char* e = std::getenv("IBR_SMOOTHER");
        return e && std::strcmp(e, "halfsweep") == 0;
    }();
    return !off && g.d == 3 && g.n0 % FX == 0 && g.n1 % FY == 0 && g.n2 >= 4 && g.ncell >= min_cells;
}

template <typename T>
void mg_sweep_fused(const Geo& g, const T* u_old, const T* f, T* u_new, int C, double sigma, double kappa, int c0,
                    bool zero_init, cudaStream_t s) {
    T kh2 = (T)(kappa / (g.h * g.h));
    dim3 grid((g.n0 / FX) * (g.n1 / FY), (g.n2 + FZ - 1) / FZ, C);
    ProfScope ps(KID_RBGS, s, (zero_init ? 2.0 : 3.0) * C * g.ncell * sizeof(T));
    k_rbgs_fused3d<T><<<grid, FX * FY, 0, s>>>(u_old, f, u_new, g, (T)sigma, kh2, c0, zero_init ? 1 : 0);
    IBR_CHECK_LAUNCH();
}

template <typename T>
void mg_residual_restrict(const Geo& gf, const Geo& gc, const T* u, const T* f, T* fc, int C, double sigma,
                          double kappa, cudaStream_t s) {
    T kh2 = (T)(kappa / (gf.h * gf.h));
    dim3 grid(grid_1d(gc.ncell, 256), C);
    ProfScope ps(KID_RESTRICT, s, (2.0 * gf.ncell + gc.ncell) * C * sizeof(T));
    if (gf.d == 3)
        k_resid_restrict<3, T><<<grid, 256, 0, s>>>(u, f, fc, gf, gc, (T)sigma, kh2);
    else
        k_resid_restrict<2, T><<<grid, 256, 0, s>>>(u, f, fc, gf, gc, (T)sigma, kh2);
    IBR_CHECK_LAUNCH();
}

template <typename T>
void mg_prolong_correct(const Geo& gf, const Geo& gc, T* u, const T* uc, int C, cudaStream_t s) {
    dim3 grid(grid_1d(gf.ncell, 256), C);
    ProfScope ps(KID_PROLONG, s, (2.0 * gf.ncell + gc.ncell) * C * sizeof(T));
    if (gf.d == 3)
        k_prolong<3, T><<<grid, 256, 0, s>>>(u, uc, gf, gc);
    else
        k_prolong<2, T><<<grid, 256, 0, s>>>(u, uc, gf, gc);
    IBR_CHECK_LAUNCH();
}

template <typename T>
void mg_coarse_solve(const Geo& g, T* u, const T* f, int C, double sigma, double kappa, int sweeps,
                     cudaStream_t s) {
    T kh2 = (T)(kappa / (g.h * g.h));
    size_t sm = 2 * (size_t)g.ncell * sizeof(T);
    int nt = g.ncell >= 1024 ? 1024 : (int)((g.ncell + 31) / 32 * 32);
    ProfScope ps(KID_COARSE, s, 2.0 * C * g.ncell * sizeof(T));
    if (g.d == 3)
        k_coarse<3, T><<<C, nt, sm, s>>>(u, f, g, (T)sigma, kh2, sweeps);
    else
        k_coarse<2, T><<<C, nt, sm, s>>>(u, f, g, (T)sigma, kh2, sweeps);
    IBR_CHECK_LAUNCH();
}

template <typename T>
void ps_divergence(const Geo& g, const T* y, const T* hd, T* q_rhs, double rhs_scale, T* q, cudaStream_t s) {
    int nb = grid_1d(g.ncell, 256);
    ProfScope ps(KID_PS_DIV, s, (g.d + 3.0) * g.ncell * sizeof(T));
    if (g.d == 3)
        k_ps_div<3, T><<<nb, 256, 0, s>>>(y, hd, q_rhs, (T)rhs_scale, q, g, (T)(1.0 / g.h));
    else
        k_ps_div<2, T><<<nb, 256, 0, s>>>(y, hd, q_rhs, (T)rhs_scale, q, g, (T)(1.0 / g.h));
    IBR_CHECK_LAUNCH();
}

template <typename T>
void ps_finish(const Geo& g, const T* y, const T* phi, const T* q, T* z, double c_q, double c_phi,
               cudaStream_t s) {
    int nb = grid_1d(g.ncell, 256);
    ProfScope ps(KID_PS_FINISH, s, (2.0 * g.d + 3.0) * g.ncell * sizeof(T));
    if (g.d == 3)
        k_ps_finish<3, T><<<nb, 256, 0, s>>>(y, phi, q, z, g, (T)g.h, (T)c_q, (T)c_phi);
    else
        k_ps_finish<2, T><<<nb, 256, 0, s>>>(y, phi, q, z, g, (T)g.h, (T)c_q, (T)c_phi);
    IBR_CHECK_LAUNCH();
}

#define IBR_INST(T)                                                                                        \
    template void stokes_apply<T>(const Geo&, const T*, T*, double, double, const double*, cudaStream_t); \
    template void mg_smooth<T>(const Geo&, T*, const T*, int, double, double, int, bool, cudaStream_t);   \
    template void mg_sweep_fused<T>(const Geo&, const T*, const T*, T*, int, double, double, int, bool,      \
                                    cudaStream_t);                                                          \
    template void mg_residual_restrict<T>(const Geo&, const Geo&, const T*, const T*, T*, int, double,    \
                                          double, cudaStream_t);                                          \
    template void mg_prolong_correct<T>(const Geo&, const Geo&, T*, const T*, int, cudaStream_t);         \
    template void mg_coarse_solve<T>(const Geo&, T*, const T*, int, double, double, int, cudaStream_t);   \
    template void ps_divergence<T>(const Geo&, const T*, const T*, T*, double, T*, cudaStream_t);         \
    template void ps_finish<T>(const Geo&, const T*, const T*, const T*, T*, double, double, cudaStream_t);
IBR_INST(double)
IBR_INST(float)
#undef IBR_INST

}  // namespace ibr
