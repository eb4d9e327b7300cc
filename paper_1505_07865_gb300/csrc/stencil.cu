// MAC-grid operators and the geometric multigrid pieces of P_S (Sec. V.B).
//
// Layout: a scalar field is ncell values, x fastest; a stack of C fields is
// C*ncell values.  A Stokes vector is [v_0 .. v_{d-1} | p].  Every axis has an
// even number of cells (red-black ordering).  An axis is periodic, or bounded
// by walls (App. D).  Beyond a wall a field is extended by linear
// extrapolation through the wall value; for the homogeneous operators here:
//   velocity tangential to the wall (cell-centred along the axis): ghost = -u
//   pressure: ghost = +u (homogeneous Neumann)
//   normal velocity: faces 0..n, face 0 stored as a boundary entry (identity
//   row), face n not stored; both wall faces add nothing to their neighbours.
// The kernels are templated on W (some axis has walls); the W = false
// instances are the plain wrapped stencils.  Boundary data enters only the
// right-hand side (wall_lift).
#include <algorithm>
#include <array>
#include <cstdlib>
#include <iterator>
#include <map>
#include <mutex>
#include <vector>

#include <cooperative_groups.h>

#include "ibr_internal.cuh"

namespace cg = cooperative_groups;

namespace ibr {
namespace {

// Division of non-negative 32-bit indices (n < 2^31) by a divisor fixed per
// launch, by a multiply-high and a shift (Granlund and Montgomery, "Division by
// invariant integers using multiplication", 1994): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, n / d = (umulhi(m, n) + n) >> l.
struct FastDiv {
    unsigned m;
    int l;
};
FastDiv make_fastdiv(unsigned d) {
    int l = 0;
    while ((1ULL << l) < d) ++l;
    FastDiv f;
    f.m = (unsigned)(((1ULL << 32) * ((1ULL << l) - d)) / d + 1);
    f.l = l;
    return f;
}
__device__ __forceinline__ int fdiv(int n, FastDiv f) {
    return (int)((__umulhi(f.m, (unsigned)n) + (unsigned)n) >> f.l);
}

// flat index and wrapped neighbour offsets of a cell; 32-bit (a field has
// fewer than 2^31 cells, checked when the grid is created)
struct Nbr {
    int c;
    int xp, xm;
    int yp, ym;
    int zp, zm;
};

template <int D>
__device__ __forceinline__ Nbr neighbours(const Geo& g, int i, int j, int k) {
    Nbr n;
    const int sy = g.n0;
    const int sz = g.n0 * g.n1;
    n.c = i + sy * j + sz * k;
    n.xp = (i == g.n0 - 1) ? 1 - g.n0 : 1;
    n.xm = (i == 0) ? g.n0 - 1 : -1;
    n.yp = (j == g.n1 - 1) ? (1 - g.n1) * sy : sy;
    n.ym = (j == 0) ? (g.n1 - 1) * sy : -sy;
    if (D == 3) {
        n.zp = (k == g.n2 - 1) ? (1 - g.n2) * sz : sz;
        n.zm = (k == 0) ? (g.n2 - 1) * sz : -sz;
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

// Boundary rule of field fld at cell (i, j, k) on the wall axes.
// ok bit 2a (2a+1): the low (high) neighbour along a is an unknown of the
// stencil; adj: change of the Laplacian's diagonal from mirror ghosts (-1 per
// Dirichlet side, +1 per Neumann side); ident: a stored wall face.
struct WInfo {
    unsigned ok;
    int adj;
    bool ident;
};

template <int D>
__device__ __forceinline__ WInfo wall_info(const Geo& g, int fld, int i, int j, int k) {
    WInfo w;
    w.ok = 0x3Fu;
    w.adj = 0;
    w.ident = false;
    const int id[3] = {i, j, k};
    const int ns[3] = {g.n0, g.n1, g.n2};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        if (!((g.wall >> a) & 1)) continue;
        const int x = id[a], n = ns[a];
        if (fld == a) {
            if (x == 0) w.ident = true;
            if (x <= 1) w.ok &= ~(1u << (2 * a));
            if (x == n - 1) w.ok &= ~(2u << (2 * a));
        } else {
            const int sgn = fld == FLD_P ? 1 : -1;
            if (x == 0) {
                w.ok &= ~(1u << (2 * a));
                w.adj += sgn;
            }
            if (x == n - 1) {
                w.ok &= ~(2u << (2 * a));
                w.adj += sgn;
            }
        }
    }
    return w;
}

template <int D, typename T>
__device__ __forceinline__ T nbr_sum_w(const T* __restrict__ u, const Nbr& n, unsigned ok) {
    T s = T(0);
    if (ok & 1u) s += u[n.c + n.xm];
    if (ok & 2u) s += u[n.c + n.xp];
    if (ok & 4u) s += u[n.c + n.ym];
    if (ok & 8u) s += u[n.c + n.yp];
    if (D == 3) {
        if (ok & 16u) s += u[n.c + n.zm];
        if (ok & 32u) s += u[n.c + n.zp];
    }
    return s;
}

// field code of the cmp-th stacked field
__device__ __forceinline__ int field_of(int fld0, int cmp) { return fld0 == FLD_P ? FLD_P : fld0 + cmp; }

// the operator of field fld has the constants as null space: sigma == 0 and
// no Dirichlet rule on any axis (the pressure, or a fully periodic grid)
__device__ __forceinline__ bool singular_field(const Geo& g, int fld, double sigma) {
    return sigma == 0.0 && (g.wall == 0 || fld == FLD_P);
}

// y_v^a = sigma v^a - kh2 Lap v^a + (p_c - p_{c-e_a}) ih + shift_a ;
// y_p = -ih sum_a (v^a_{c+e_a} - v^a_c)   (walls: wall faces add nothing,
// wall-face rows are the identity)
// Launch shape of the grid kernels: blocks of 32 x 8 threads over (x, y),
// gridDim.z = n2 * (number of stacked fields); no 64-bit index division.
constexpr int BX = 32, BY = 8;

template <int D, bool W, typename T>
__global__ void __launch_bounds__(256) k_stokes(const T* __restrict__ x, T* __restrict__ y, Geo g, T sigma, T kh2,
                                                T ih, const double* __restrict__ shift) {
    pdl_start();
    int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
    if (i >= g.n0 || j >= g.n1) return;
    Nbr n = neighbours<D>(g, i, j, k);
    const T* p = x + D * g.ncell;
    T pc = p[n.c];
    T div = T(0);
    const int pm[3] = {n.xm, n.ym, n.zm};
    const int pp[3] = {n.xp, n.yp, n.zp};
    const int id[3] = {i, j, k};
    const int ns[3] = {g.n0, g.n1, g.n2};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const T* u = x + a * g.ncell;
        T uc = u[n.c];
        T val;
        if (!W) {
            T lap = nbr_sum<D, T>(u, n) - T(2 * D) * uc;
            val = sigma * uc - kh2 * lap + (pc - p[n.c + pm[a]]) * ih;
            div += u[n.c + pp[a]] - uc;
        } else {
            WInfo wi = wall_info<D>(g, a, i, j, k);
            if (wi.ident) {
                val = uc;
            } else {
                T lap = nbr_sum_w<D, T>(u, n, wi.ok) + T(wi.adj - 2 * D) * uc;
                val = sigma * uc - kh2 * lap + (pc - p[n.c + pm[a]]) * ih;
            }
            const bool wa = (g.wall >> a) & 1;
            T hi = (wa && id[a] == ns[a] - 1) ? T(0) : u[n.c + pp[a]];
            T lo = (wa && id[a] == 0) ? T(0) : uc;
            div += hi - lo;
        }
        if (shift) val += (T)shift[a];
        y[a * g.ncell + n.c] = val;
    }
    y[D * g.ncell + n.c] = -div * ih;
}

// ---- point operators shared by the per-level kernels and the one-CTA tail ----
// (same arithmetic, so a level gives the same result on either path)

// inv_diag = 1 / (sigma + 2D kh2), formed by rbgs_inv_diag on host or device
template <int D, typename T>
__host__ __device__ __forceinline__ T rbgs_inv_diag(T sigma, T kh2) {
    T diag = sigma + T(2 * D) * kh2;
    return T(1) / diag;
}

// red-black Gauss-Seidel update of cell (i, j, k) of field fld
template <int D, bool W, typename T>
__device__ __forceinline__ void rbgs_cell(T* u, const T* f, const Geo& g, int fld, T sigma, T kh2, T inv_diag,
                                          int zero_init, int i, int j, int k) {
    Nbr n = neighbours<D>(g, i, j, k);
    if (!W) {
        T nb = zero_init ? T(0) : nbr_sum<D, T>(u, n);
        u[n.c] = (f[n.c] + kh2 * nb) * inv_diag;
    } else {
        WInfo wi = wall_info<D>(g, fld, i, j, k);
        if (wi.ident) {
            u[n.c] = f[n.c];
            return;
        }
        T nb = zero_init ? T(0) : nbr_sum_w<D, T>(u, n, wi.ok);
        T dinv = wi.adj == 0 ? inv_diag : T(1) / (sigma + kh2 * T(2 * D - wi.adj));
        u[n.c] = (f[n.c] + kh2 * nb) * dinv;
    }
}

// the same for the t-th cell of the given colour (x index ih = t mod n0/2);
// dh, d1: division by n0/2 and by n1
template <int D, bool W, typename T>
__device__ __forceinline__ void rbgs_point(T* u, const T* f, const Geo& g, int fld, T sigma, T kh2, T inv_diag,
                                           int color, int zero_init, int t, FastDiv dh, FastDiv d1) {
    const int hn0 = g.n0 >> 1;
    const int r = fdiv(t, dh);
    const int ih = t - r * hn0;
    const int k = fdiv(r, d1);
    const int j = r - k * g.n1;
    rbgs_cell<D, W, T>(u, f, g, fld, sigma, kh2, inv_diag, zero_init, 2 * ih + ((j + k + color) & 1), j, k);
}

// residual f - (sigma u - kh2 Lap u) at fine cell (i, j, k)
template <int D, bool W, typename T>
__device__ __forceinline__ T resid_cell(const T* u, const T* f, const Geo& g, int fld, T sigma, T kh2, int i, int j,
                                        int k) {
    Nbr n = neighbours<D>(g, i, j, k);
    T uc = u[n.c];
    if (!W) return f[n.c] - (sigma * uc - kh2 * (nbr_sum<D, T>(u, n) - T(2 * D) * uc));
    WInfo wi = wall_info<D>(g, fld, i, j, k);
    if (wi.ident) return f[n.c] - uc;
    return f[n.c] - (sigma * uc - kh2 * (nbr_sum_w<D, T>(u, n, wi.ok) + T(wi.adj - 2 * D) * uc));
}

// coarse cell (I, J, K): average over its 2^D children of the residual; the
// normal component on its own wall axis is vertex-centred there: full
// weighting (1/4, 1/2, 1/4) of the fine faces 2I-1, 2I, 2I+1, and zero on the
// coarse wall face I = 0
template <int D, bool W, typename T>
__device__ __forceinline__ T restrict_cell(const T* u, const T* f, const Geo& gf, int fld, T sigma, T kh2, int I,
                                           int J, int K) {
    if (!W) {
        T acc = T(0);
#pragma unroll
        for (int c = 0; c < (1 << D); ++c) {
            int i = 2 * I + (c & 1);
            int j = 2 * J + ((c >> 1) & 1);
            int k = D == 3 ? 2 * K + ((c >> 2) & 1) : 0;
            acc += resid_cell<D, false, T>(u, f, gf, fld, sigma, kh2, i, j, k);
        }
        return acc * (T(1) / T(1 << D));
    }
    const int Xc[3] = {I, J, K};
    int fi[3][3];
    T fw[3][3];
    int cnt[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a >= D) {
            cnt[a] = 1;
            fi[a][0] = 0;
            fw[a][0] = T(1);
        } else if (((gf.wall >> a) & 1) && fld == a) {
            if (Xc[a] == 0) return T(0);
            cnt[a] = 3;
            fi[a][0] = 2 * Xc[a] - 1;
            fi[a][1] = 2 * Xc[a];
            fi[a][2] = 2 * Xc[a] + 1;
            fw[a][0] = T(0.25);
            fw[a][1] = T(0.5);
            fw[a][2] = T(0.25);
        } else {
            cnt[a] = 2;
            fi[a][0] = 2 * Xc[a];
            fi[a][1] = 2 * Xc[a] + 1;
            fw[a][0] = fw[a][1] = T(0.5);
        }
    }
    T acc = T(0);
    for (int p = 0; p < cnt[0]; ++p)
        for (int q = 0; q < cnt[1]; ++q)
            for (int r = 0; r < cnt[2]; ++r)
                acc += fw[0][p] * fw[1][q] * fw[2][r] *
                       resid_cell<D, true, T>(u, f, gf, fld, sigma, kh2, fi[0][p], fi[1][q], fi[2][r]);
    return acc;
}

template <int D, bool W, typename T>
__device__ __forceinline__ T restrict_point(const T* u, const T* f, const Geo& gf, const Geo& gc, int fld, T sigma,
                                            T kh2, int t, FastDiv dc0, FastDiv dc1) {
    const int r = fdiv(t, dc0);
    const int I = t - r * gc.n0;
    const int K = fdiv(r, dc1);
    const int J = r - K * gc.n1;
    return restrict_cell<D, W, T>(u, f, gf, fld, sigma, kh2, I, J, K);
}

// fine cell (i, j, k): cell-centred (bi/tri)linear interpolation of the coarse
// correction, weights 3/4 (parent) and 1/4 (the neighbour on the child's
// side; beyond a wall the mirror ghost of the parent, -/+ for Dirichlet /
// Neumann).  The normal component on its own wall axis: injection at even
// faces, the mean of the two coarse faces at odd ones, wall faces zero.
template <int D, bool W, typename T>
__device__ __forceinline__ T prolong_cell(const T* cc, const Geo& gc, int fld, int i, int j, int k) {
    if (!W) {
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
            int idx = I[a] + gc.n0 * (Jc[b] + gc.n1 * Kc[e]);
            acc += ww * cc[idx];
        }
        return acc;
    }
    const int id[3] = {i, j, k};
    const int nc[3] = {gc.n0, gc.n1, gc.n2};
    int ci[3][2];
    T cw[3][2];
    int cnt[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a >= D) {
            cnt[a] = 1;
            ci[a][0] = 0;
            cw[a][0] = T(1);
            continue;
        }
        const int x = id[a], X = x >> 1;
        const bool wa = (gc.wall >> a) & 1;
        if (!wa) {
            cnt[a] = 2;
            ci[a][0] = X;
            cw[a][0] = T(0.75);
            ci[a][1] = (x & 1) ? (X + 1 == nc[a] ? 0 : X + 1) : (X == 0 ? nc[a] - 1 : X - 1);
            cw[a][1] = T(0.25);
        } else if (fld == a) {
            if ((x & 1) == 0) {
                cnt[a] = 1;
                ci[a][0] = X;
                cw[a][0] = X == 0 ? T(0) : T(1);
            } else {
                cnt[a] = 2;
                ci[a][0] = X;
                cw[a][0] = X == 0 ? T(0) : T(0.5);
                ci[a][1] = X + 1 == nc[a] ? 0 : X + 1;
                cw[a][1] = X + 1 == nc[a] ? T(0) : T(0.5);
            }
        } else {
            cnt[a] = 2;
            ci[a][0] = X;
            cw[a][0] = T(0.75);
            const int nb = (x & 1) ? X + 1 : X - 1;
            if (nb < 0 || nb >= nc[a]) {
                ci[a][1] = X;
                cw[a][1] = fld == FLD_P ? T(0.25) : T(-0.25);
            } else {
                ci[a][1] = nb;
                cw[a][1] = T(0.25);
            }
        }
    }
    T acc = T(0);
    for (int p = 0; p < cnt[0]; ++p)
        for (int q = 0; q < cnt[1]; ++q)
            for (int r = 0; r < cnt[2]; ++r)
                acc += cw[0][p] * cw[1][q] * cw[2][r] * cc[ci[0][p] + gc.n0 * (ci[1][q] + gc.n1 * ci[2][r])];
    return acc;
}

template <int D, bool W, typename T>
__device__ __forceinline__ T prolong_point(const T* cc, const Geo& gf, const Geo& gc, int fld, int t, FastDiv df0,
                                           FastDiv df1) {
    const int r = fdiv(t, df0);
    const int i = t - r * gf.n0;
    const int k = fdiv(r, df1);
    const int j = r - k * gf.n1;
    return prolong_cell<D, W, T>(cc, gc, fld, i, j, k);
}

// block-wide mean of a[0..n) (all threads get it); red: 32 doubles of shared memory
template <typename T>
__device__ double block_mean(const T* a, int n, double* red) {
    int tid = threadIdx.x, nt = blockDim.x;
    double part = 0.0;
    for (int c = tid; c < n; c += nt) part += (double)a[c];
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
    double m = red[0] / (double)n;
    __syncthreads();
    return m;
}

// coarsest-level solve in shared memory: for a singular field f (in sf,
// modified) is made mean-free, u (su) from zero by red-black sweeps, then made
// mean-free; d0, d1: division by n0 and n1
template <int D, bool W, typename T>
__device__ void coarse_block(T* su, T* sf, const Geo& g, int fld, T sigma, T kh2, T inv, int sweeps, double* red,
                             FastDiv d0, FastDiv d1) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int nc = (int)g.ncell;
    const bool sing = singular_field(g, fld, (double)sigma);
    T fmean = sing ? (T)block_mean(sf, nc, red) : T(0);
    for (int c = tid; c < nc; c += nt) {
        sf[c] -= fmean;
        su[c] = T(0);
    }
    __syncthreads();
    for (int s = 0; s < sweeps; ++s) {
        for (int color = 0; color < 2; ++color) {
            for (int c = tid; c < nc; c += nt) {
                const int r = fdiv(c, d0);
                const int i = c - r * g.n0;
                const int k = fdiv(r, d1);
                const int j = r - k * g.n1;
                if (((i + j + k) & 1) != color) continue;
                rbgs_cell<D, W, T>(su, sf, g, fld, sigma, kh2, inv, 0, i, j, k);
            }
            __syncthreads();
        }
    }
    T umean = sing ? (T)block_mean(su, nc, red) : T(0);
    for (int c = tid; c < nc; c += nt) su[c] -= umean;
    __syncthreads();
}

// red-black Gauss-Seidel half sweep on C stacked fields (component from blockIdx.z)
template <int D, bool W, typename T>
__global__ void __launch_bounds__(256) k_rbgs(T* __restrict__ u, const T* __restrict__ f, Geo g, int fld0, T sigma,
                                              T kh2, T inv_diag, int color, int zero_init) {
    pdl_start();
    int ih = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    int k = blockIdx.z % g.n2, cmp = blockIdx.z / g.n2;
    if (ih >= (g.n0 >> 1) || j >= g.n1) return;
    long long off = (long long)cmp * g.ncell;
    rbgs_cell<D, W, T>(u + off, f + off, g, field_of(fld0, cmp), sigma, kh2, inv_diag, zero_init,
                       2 * ih + ((j + k + color) & 1), j, k);
}

// the same half sweep on a periodic 3-D grid, each thread a column of kz
// cells along z at fixed (ih, j): the y wrap and the block decomposition
// are paid once per column, the cells of a column are independent (one
// colour) so their loads overlap.  Same arithmetic and summation order as
// rbgs_cell, so the result is bitwise that of k_rbgs, whatever the tile
// (32 x by threads, kz cells each; picked per level shape by the tuner).
template <typename T>
__global__ void __launch_bounds__(256) k_rbgs_col(T* __restrict__ u, const T* __restrict__ f, Geo g, int nkb, int kz,
                                                  T kh2, T inv_diag, int color, int zero_init) {
    pdl_start();
    const int ih = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    const int cmp = blockIdx.z / nkb, kb = blockIdx.z - cmp * nkb;
    if (ih >= (g.n0 >> 1) || j >= g.n1) return;
    const long long off = (long long)cmp * g.ncell;
    u += off;
    f += off;
    const int n0 = g.n0, n1 = g.n1, n2 = g.n2;
    const int sy = n0, sz = n0 * n1;
    const int yp = (j == n1 - 1) ? (1 - n1) * sy : sy;
    const int ym = (j == 0) ? (n1 - 1) * sy : -sy;
    const int k0 = kb * kz, k1 = min(k0 + kz, n2);
#pragma unroll 4
    for (int k = k0; k < k1; ++k) {
        const int i = 2 * ih + ((j + k + color) & 1);
        const int c = i + sy * j + sz * k;
        const int xp = (i == n0 - 1) ? 1 - n0 : 1;
        const int xm = (i == 0) ? n0 - 1 : -1;
        const int zp = (k == n2 - 1) ? (1 - n2) * sz : sz;
        const int zm = (k == 0) ? (n2 - 1) * sz : -sz;
        T nb = T(0);
        if (!zero_init) {
            nb = u[c + xp] + u[c + xm] + u[c + yp] + u[c + ym];
            nb += u[c + zp] + u[c + zm];
        }
        u[c] = (f[c] + kh2 * nb) * inv_diag;
    }
}

template <int D, bool W, typename T>
__global__ void __launch_bounds__(256) k_resid_restrict(const T* __restrict__ u, const T* __restrict__ f,
                                                        T* __restrict__ fc, Geo gf, Geo gc, int fld0, T sigma,
                                                        T kh2) {
    pdl_start();
    int I = blockIdx.x * BX + threadIdx.x, J = blockIdx.y * BY + threadIdx.y;
    int K = blockIdx.z % gc.n2, cmp = blockIdx.z / gc.n2;
    if (I >= gc.n0 || J >= gc.n1) return;
    long long t = I + (long long)gc.n0 * (J + (long long)gc.n1 * K);
    fc[cmp * gc.ncell + t] = restrict_cell<D, W, T>(u + cmp * gf.ncell, f + cmp * gf.ncell, gf,
                                                    field_of(fld0, cmp), sigma, kh2, I, J, K);
}

template <int D, bool W, typename T>
__global__ void __launch_bounds__(256) k_prolong(T* __restrict__ u, const T* __restrict__ uc, Geo gf, Geo gc,
                                                 int fld0) {
    pdl_start();
    int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
    int k = blockIdx.z % gf.n2, cmp = blockIdx.z / gf.n2;
    if (i >= gf.n0 || j >= gf.n1) return;
    long long t = i + (long long)gf.n0 * (j + (long long)gf.n1 * k);
    u[cmp * gf.ncell + t] += prolong_cell<D, W, T>(uc + cmp * gc.ncell, gc, field_of(fld0, cmp), i, j, k);
}

// single-CTA coarse solve of the coarsest level (one CTA per field)
template <int D, bool W, typename T>
__global__ void __launch_bounds__(1024) k_coarse(T* __restrict__ u, const T* __restrict__ f, Geo g, int fld0,
                                                 T sigma, T kh2, T inv, int sweeps, FastDiv d0, FastDiv d1) {
    extern __shared__ unsigned char smem_raw[];
    T* su = reinterpret_cast<T*>(smem_raw);
    T* sf = su + g.ncell;
    __shared__ double red[32];
    int cmp = blockIdx.x;
    const T* ff = f + cmp * g.ncell;
    T* uu = u + cmp * g.ncell;
    for (int c = threadIdx.x; c < (int)g.ncell; c += blockDim.x) sf[c] = ff[c];
    __syncthreads();
    coarse_block<D, W, T>(su, sf, g, field_of(fld0, cmp), sigma, kh2, inv, sweeps, red, d0, d1);
    for (int c = threadIdx.x; c < (int)g.ncell; c += blockDim.x) uu[c] = su[c];
}

// The small levels of a V-cycle, all in one CTA's shared memory (one CTA per
// field): levels tl.g[0] (finest of the tail) .. tl.g[nl-1] (coarsest), the
// same sweeps, restriction, coarse solve and prolongation as the per-level
// kernels, with __syncthreads between them instead of kernel launches.
// Index arithmetic in 32 bits with the per-level divisors precomputed.
struct TailLevels {
    int nl;
    Geo g[MG_TAIL_MAX_LEVELS];
    int uoff[MG_TAIL_MAX_LEVELS];
    int foff[MG_TAIL_MAX_LEVELS];
    FastDiv dh[MG_TAIL_MAX_LEVELS];  // n0 / 2
    FastDiv d0[MG_TAIL_MAX_LEVELS];  // n0
    FastDiv d1[MG_TAIL_MAX_LEVELS];  // n1
    // per level kappa h^-2 and the smoother's 1 / (sigma + 2D kappa h^-2),
    // formed on the host in the kernels' precision (FP64 arithmetic runs at
    // 1/64 of the FP32 rate on this part: no per-thread FP64 division)
    float kh2f[MG_TAIL_MAX_LEVELS], invf[MG_TAIL_MAX_LEVELS];
    double kh2d[MG_TAIL_MAX_LEVELS], invd[MG_TAIL_MAX_LEVELS];
};

template <typename T, typename L>
__device__ __forceinline__ T lev_kh2(const L& tl, int l) {
    if constexpr (sizeof(T) == 4) return tl.kh2f[l]; else return tl.kh2d[l];
}
template <typename T, typename L>
__device__ __forceinline__ T lev_inv(const L& tl, int l) {
    if constexpr (sizeof(T) == 4) return tl.invf[l]; else return tl.invd[l];
}

// the V-cycle over the levels of tl, whose finest level's f (and u unless
// zero_start) are already in shared memory at sm; leaves u of the finest
// level there.  Every thread of the CTA calls it.
template <int D, bool W, typename T>
__device__ void tail_solve(const TailLevels& tl, T* sm, int fld, T sigma, int zero_start, int pre, int post,
                           int sweeps, double* red) {
    const int tid = threadIdx.x, nt = blockDim.x;
    auto half = [&](int l, int color, int zero) {
        const Geo& g = tl.g[l];
        const T kh2 = lev_kh2<T>(tl, l);
        const T inv = lev_inv<T>(tl, l);
        T* u = sm + tl.uoff[l];
        const T* f = sm + tl.foff[l];
        const int np = (int)(g.ncell >> 1);
        for (int t = tid; t < np; t += nt)
            rbgs_point<D, W, T>(u, f, g, fld, sigma, kh2, inv, color, zero, t, tl.dh[l], tl.d1[l]);
        __syncthreads();
    };
    const int L = tl.nl;
    if (L == 1) {
        const Geo& g = tl.g[0];
        if (zero_start) {
            coarse_block<D, W, T>(sm + tl.uoff[0], sm + tl.foff[0], g, fld, sigma, lev_kh2<T>(tl, 0),
                                  lev_inv<T>(tl, 0), sweeps, red, tl.d0[0], tl.d1[0]);
        } else {
            for (int s = 0; s < sweeps; ++s) {
                half(0, 0, 0);
                half(0, 1, 0);
            }
        }
        return;
    }
    for (int l = 0; l + 1 < L; ++l) {
        int zs = (l > 0) || zero_start;
        if (pre == 0 && zs) {
            T* u = sm + tl.uoff[l];
            for (int c = tid; c < (int)tl.g[l].ncell; c += nt) u[c] = T(0);
            __syncthreads();
        }
        for (int it = 0; it < pre; ++it) {
            half(l, 0, zs && it == 0);
            half(l, 1, 0);
        }
        const Geo& gf = tl.g[l];
        const Geo& gc = tl.g[l + 1];
        const T kh2 = lev_kh2<T>(tl, l);
        const T* u = sm + tl.uoff[l];
        const T* f = sm + tl.foff[l];
        T* fc = sm + tl.foff[l + 1];
        for (int t = tid; t < (int)gc.ncell; t += nt)
            fc[t] = restrict_point<D, W, T>(u, f, gf, gc, fld, sigma, kh2, t, tl.d0[l + 1], tl.d1[l + 1]);
        __syncthreads();
    }
    {
        const Geo& g = tl.g[L - 1];
        coarse_block<D, W, T>(sm + tl.uoff[L - 1], sm + tl.foff[L - 1], g, fld, sigma, lev_kh2<T>(tl, L - 1),
                              lev_inv<T>(tl, L - 1), sweeps, red, tl.d0[L - 1], tl.d1[L - 1]);
    }
    for (int l = L - 2; l >= 0; --l) {
        const Geo& gf = tl.g[l];
        const Geo& gc = tl.g[l + 1];
        T* u = sm + tl.uoff[l];
        const T* uc = sm + tl.uoff[l + 1];
        for (int t = tid; t < (int)gf.ncell; t += nt)
            u[t] += prolong_point<D, W, T>(uc, gf, gc, fld, t, tl.d0[l], tl.d1[l]);
        __syncthreads();
        for (int it = 0; it < post; ++it) {
            half(l, 1, 0);
            half(l, 0, 0);
        }
    }
}

template <int D, bool W, typename T>
__global__ void __launch_bounds__(1024) k_mg_tail(const __grid_constant__ TailLevels tl, T* __restrict__ ug,
                                                  const T* __restrict__ fg,
                                                  int fld0, T sigma, int zero_start, int pre, int post,
                                                  int sweeps) {
    pdl_start();
    extern __shared__ unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    __shared__ double red[32];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int cmp = blockIdx.x;
    const int fld = field_of(fld0, cmp);
    const int n0 = (int)tl.g[0].ncell;
    ug += (long long)cmp * n0;
    fg += (long long)cmp * n0;
    {
        T* u0 = sm + tl.uoff[0];
        T* f0 = sm + tl.foff[0];
        for (int c = tid; c < n0; c += nt) {
            f0[c] = fg[c];
            u0[c] = zero_start ? T(0) : ug[c];
        }
    }
    __syncthreads();
    tail_solve<D, W, T>(tl, sm, fld, sigma, zero_start, pre, post, sweeps, red);
    {
        const T* u0 = sm + tl.uoff[0];
        for (int c = tid; c < n0; c += nt) ug[c] = u0[c];
    }
}

// ---- the finest level of a periodic 3-D V-cycle in red-black split layout ----
// During the V-cycle the finest level's u and f live in two arrays per
// stacked field, one per colour: cell (i, j, k) of colour c = (i+j+k) & 1 at
// index (i >> 1) + (n0/2) (j + n1 k) of colour array c (field q, colour c at
// offset (2q + c) n/2).  A half sweep then reads the other colour's cells
// contiguously (its x-neighbours are entries ih + p - 1 and ih + p of the
// same row, p = (j+k+c) & 1; its y- and z-neighbours entry ih of rows j+-1
// and planes k+-1), so every sector it loads is used, four cells per thread.
// The conversion from and to the natural layout is folded into the first
// (zero-start) and the last half sweep.  Same arithmetic and summation order
// as rbgs_cell / resid_cell / prolong_cell: bitwise the same V-cycle.
constexpr int RB_V = 4;  // cells of one colour per thread (n0 % 8 == 0)

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
    using type = float4;
};
template <>
struct Vec4<double> {
    using type = double4;
};

template <typename T>
__device__ __forceinline__ void ld4(const T* p, T (&v)[4]) {
    const typename Vec4<T>::type x = *reinterpret_cast<const typename Vec4<T>::type*>(p);
    v[0] = x.x;
    v[1] = x.y;
    v[2] = x.z;
    v[3] = x.w;
}
template <typename T>
__device__ __forceinline__ void st4(T* p, const T (&v)[4]) {
    typename Vec4<T>::type x;
    x.x = v[0];
    x.y = v[1];
    x.z = v[2];
    x.w = v[3];
    *reinterpret_cast<typename Vec4<T>::type*>(p) = x;
}

// thread -> (field q, plane k, row j, first entry ih of its RB_V entries)
struct RbIdx {
    int q, k, j, ih;
};
__device__ __forceinline__ RbIdx rb_index(int t, int hq, FastDiv dq, int n1, FastDiv d1, int n2, FastDiv d2) {
    RbIdx r;
    const int row = fdiv(t, dq);
    r.ih = (t - row * hq) * RB_V;
    const int kk = fdiv(row, d1);
    r.j = row - kk * n1;
    r.q = fdiv(kk, d2);
    r.k = kk - r.q * n2;
    return r;
}

// the first (zero-start) half sweep of colour 0 from the natural f: writes
// both colours of f into the split arrays and u_0 = f_0 / diag
template <typename T>
__global__ void __launch_bounds__(256) k_rb_first(const T* __restrict__ fnat, T* __restrict__ fs, T* __restrict__ us,
                                                  int n0, int n1, int n2, int nthreads, FastDiv dq, FastDiv d1,
                                                  FastDiv d2, T inv) {
    pdl_start();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nthreads) return;
    const int hn = n0 >> 1, hq = hn / RB_V;
    const RbIdx r = rb_index(t, hq, dq, n1, d1, n2, d2);
    const long long half = (long long)hn * n1 * n2;
    const long long rowoff = (long long)hn * (r.j + (long long)n1 * r.k) + r.ih;
    const T* src = fnat + (long long)r.q * 2 * half + ((long long)n0 * (r.j + (long long)n1 * r.k) + 2 * r.ih);
    T a[4], b[4];
    ld4(src, a);
    ld4(src + 4, b);
    const T nat[8] = {a[0], a[1], a[2], a[3], b[0], b[1], b[2], b[3]};
    const bool p0 = ((r.j + r.k) & 1) != 0;  // x offset of colour 0 in this row
    T c0[4], c1[4], u0[4];
#pragma unroll
    for (int e = 0; e < RB_V; ++e) {
        c0[e] = p0 ? nat[2 * e + 1] : nat[2 * e];
        c1[e] = p0 ? nat[2 * e] : nat[2 * e + 1];
        u0[e] = c0[e] * inv;  // the zero-start update (f + kappa h^-2 0) / diag
    }
    T* f0 = fs + (long long)(2 * r.q) * half;
    T* f1 = f0 + half;
    st4(f0 + rowoff, c0);
    st4(f1 + rowoff, c1);
    st4(us + (long long)(2 * r.q) * half + rowoff, u0);
}

// half sweep of colour c in split layout; last != 0: also writes both
// colours of u to the natural array unat (the V-cycle's output)
template <typename T>
__global__ void __launch_bounds__(256) k_rb_half(T* __restrict__ us, const T* __restrict__ fs, int n0, int n1, int n2,
                                                 int nthreads, FastDiv dq, FastDiv d1, FastDiv d2, T kh2, T inv,
                                                 int color, T* __restrict__ unat) {
    pdl_start();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nthreads) return;
    const int hn = n0 >> 1, hq = hn / RB_V;
    const RbIdx r = rb_index(t, hq, dq, n1, d1, n2, d2);
    const long long half = (long long)hn * n1 * n2;
    T* dst = us + (long long)(2 * r.q + color) * half;
    const T* src = us + (long long)(2 * r.q + 1 - color) * half;
    const T* f = fs + (long long)(2 * r.q + color) * half;
    const int p = (r.j + r.k + color) & 1;
    const long long plane = (long long)hn * n1;
    const long long row = (long long)hn * (r.j + (long long)n1 * r.k);
    const long long rym = (long long)hn * ((r.j == 0 ? n1 - 1 : r.j - 1) + (long long)n1 * r.k);
    const long long ryp = (long long)hn * ((r.j == n1 - 1 ? 0 : r.j + 1) + (long long)n1 * r.k);
    const long long rzm = row + (r.k == 0 ? (long long)(n2 - 1) * plane : -plane);
    const long long rzp = row + (r.k == n2 - 1 ? -(long long)(n2 - 1) * plane : plane);
    T cen[4], ym[4], yp[4], zm[4], zp[4], ff[4];
    ld4(src + row + r.ih, cen);
    ld4(src + rym + r.ih, ym);
    ld4(src + ryp + r.ih, yp);
    ld4(src + rzm + r.ih, zm);
    ld4(src + rzp + r.ih, zp);
    ld4(f + row + r.ih, ff);
    // the entry beyond the four: ih - 1 (p = 0) or ih + 4 (p = 1), wrapped in the row
    const int ex = p == 0 ? (r.ih == 0 ? hn - 1 : r.ih - 1) : (r.ih + RB_V == hn ? 0 : r.ih + RB_V);
    const T xe = src[row + ex];
    T out[4];
#pragma unroll
    for (int e = 0; e < RB_V; ++e) {
        // cell i = 2 (ih + e) + p: x+1 -> entry ih+e+p, x-1 -> entry ih+e+p-1
        T xp, xm;
        if (p == 0) {
            xp = cen[e];
            xm = e == 0 ? xe : cen[e - 1];
        } else {
            xp = e == RB_V - 1 ? xe : cen[e + 1];
            xm = cen[e];
        }
        T nb = xp + xm + yp[e] + ym[e];
        nb += zp[e] + zm[e];
        out[e] = (ff[e] + kh2 * nb) * inv;
    }
    st4(dst + row + r.ih, out);
    if (unat) {
        // colour c at x = 2 (ih+e) + p, the other colour (unchanged) at 2 (ih+e) + 1 - p
        T* o = unat + (long long)r.q * 2 * half + ((long long)n0 * (r.j + (long long)n1 * r.k) + 2 * r.ih);
        if (p == 0) {
            const T a[4] = {out[0], cen[0], out[1], cen[1]};
            const T b[4] = {out[2], cen[2], out[3], cen[3]};
            st4(o, a);
            st4(o + 4, b);
        } else {
            const T a[4] = {cen[0], out[0], cen[1], out[1]};
            const T b[4] = {cen[2], out[2], cen[3], out[3]};
            st4(o, a);
            st4(o + 4, b);
        }
    }
}

// coarse f = the averaged residual of the split finest level (resid_cell's
// arithmetic and the restriction's child order: bitwise the natural
// kernel's); one thread per coarse cell.  A child row (j, k) holds the
// children 2I (colour p = (j+k) & 1, entry I of colour array p) and 2I+1
// (entry I of array 1-p); their x-neighbours are entries I-1 of array 1-p
// and I+1 of array p; the y- and z-neighbours entry I of the adjacent rows,
// in the array of the other colour.  32-bit index arithmetic.
template <typename T>
__global__ void __launch_bounds__(256) k_rb_restrict(const T* __restrict__ us, const T* __restrict__ fs,
                                                     T* __restrict__ fc, int n0, int n1, int n2, int C, T sigma,
                                                     T kh2, FastDiv dc0, FastDiv dc1, FastDiv dc2) {
    pdl_start();
    const int nc0 = n0 >> 1, nc1 = n1 >> 1, nc2 = n2 >> 1;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int ncc = nc0 * nc1 * nc2;
    if (t >= ncc * C) return;
    const int r = fdiv(t, dc0);
    const int I = t - r * nc0;
    const int kk = fdiv(r, dc1);
    const int J = r - kk * nc1;
    const int q = fdiv(kk, dc2);
    const int K = kk - q * nc2;
    const int hn = nc0;  // split row length n0 / 2
    const long long half = (long long)hn * n1 * n2;
    const T* ua[2] = {us + (long long)(2 * q) * half, us + (long long)(2 * q + 1) * half};
    const T* fa[2] = {fs + (long long)(2 * q) * half, fs + (long long)(2 * q + 1) * half};
    const int Im = I == 0 ? hn - 1 : I - 1, Ip = I + 1 == hn ? 0 : I + 1;
    auto rowoff = [&](int j, int k) -> int {
        j = j < 0 ? j + n1 : (j >= n1 ? j - n1 : j);
        k = k < 0 ? k + n2 : (k >= n2 ? k - n2 : k);
        return hn * (j + n1 * k);
    };
    T acc = T(0);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int a = c & 1, j = 2 * J + ((c >> 1) & 1), k = 2 * K + ((c >> 2) & 1);
        const int col = (a + j + k) & 1;  // this child's colour; its neighbours are in array 1 - col
        const T* un = ua[1 - col];
        const int ro = rowoff(j, k);
        const T uc = ua[col][ro + I];
        // x+1, x-1: child 2I -> entries I (2I+1) and I-1 (2I-1); child 2I+1 -> I+1 (2I+2) and I (2I)
        const T xp = un[ro + (a ? Ip : I)];
        const T xm = un[ro + (a ? I : Im)];
        T nbs = xp + xm + un[rowoff(j + 1, k) + I] + un[rowoff(j - 1, k) + I];
        nbs += un[rowoff(j, k + 1) + I] + un[rowoff(j, k - 1) + I];
        const T fv = fa[col][ro + I];
        acc += fv - (sigma * uc - kh2 * (nbs - T(6) * uc));
    }
    fc[t] = acc * (T(1) / T(8));
}

// split finest u of colour 0 += the (tri)linear prolongation of the natural
// coarse u (prolong_cell's weights and order).  Only colour 0: the next
// operation, a colour-1 half sweep, overwrites every colour-1 value without
// reading it, so correcting them would change nothing.  Four cells per thread.
template <typename T>
__global__ void __launch_bounds__(256) k_rb_prolong(T* __restrict__ us, const T* __restrict__ uc, int n0, int n1,
                                                    int n2, int nthreads, FastDiv dq, FastDiv d1, FastDiv d2) {
    pdl_start();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nthreads) return;
    const int hn = n0 >> 1, hq = hn / RB_V;
    const RbIdx rr = rb_index(t, hq, dq, n1, d1, n2, d2);
    const int nc0 = n0 >> 1, nc1 = n1 >> 1, nc2 = n2 >> 1;
    const T* cc = uc + (long long)rr.q * nc0 * nc1 * nc2;
    const int j = rr.j, k = rr.k;
    const int p0 = (j + k) & 1;  // colour-0 cells of this row at x = 2 ih + p0
    int Jc[2], Kc[2];
    Jc[0] = j >> 1;
    Jc[1] = (j & 1) ? (Jc[0] + 1 == nc1 ? 0 : Jc[0] + 1) : (Jc[0] == 0 ? nc1 - 1 : Jc[0] - 1);
    Kc[0] = k >> 1;
    Kc[1] = (k & 1) ? (Kc[0] + 1 == nc2 ? 0 : Kc[0] + 1) : (Kc[0] == 0 ? nc2 - 1 : Kc[0] - 1);
    const T w[2] = {T(0.75), T(0.25)};
    const long long half = (long long)hn * n1 * n2;
    T* dst = us + (long long)(2 * rr.q) * half + (long long)hn * (j + (long long)n1 * k) + rr.ih;
    T v[4];
    ld4(dst, v);
#pragma unroll
    for (int e4 = 0; e4 < RB_V; ++e4) {
        const int ih = rr.ih + e4;  // fine x = 2 ih + p0: parent I = ih, neighbour ih + 1 (p0 = 1) or ih - 1
        int I[2];
        I[0] = ih;
        I[1] = p0 ? (ih + 1 == nc0 ? 0 : ih + 1) : (ih == 0 ? nc0 - 1 : ih - 1);
        T acc = T(0);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int a = c & 1, b = (c >> 1) & 1, e = (c >> 2) & 1;
            const T ww = w[a] * w[b] * w[e];
            acc += ww * cc[I[a] + nc0 * (Jc[b] + nc1 * Kc[e])];
        }
        v[e4] += acc;
    }
    st4(dst, v);
}

// ---- the coarse levels of a periodic 3-D V-cycle on one thread-block cluster ----
// One cluster of MG_CL CTAs per stacked field runs levels cl.top .. of the
// V-cycle in one launch.  The "distributed" levels (the first cl.nd) are split
// into z-slabs of P = n2 / MG_CL planes, CTA r of the cluster keeping planes
// [r P, (r+1) P) of u (and of f, except on the top level, whose f is read
// from global memory) in its shared memory; a cell's neighbours in the planes
// of the adjacent CTAs are read from their shared memory (distributed shared
// memory).  The remaining small levels (the tail) live in CTA 0's shared
// memory and run there (tail_solve) while the other CTAs wait.  Cluster
// barriers separate the phases.  Same point arithmetic, summation order and
// sweep order as the per-level kernels (k_rbgs_col, k_resid_restrict,
// k_prolong) and the tail.
constexpr int MG_CL = 8;
constexpr int MG_CL_MAX_LEVELS = 6;

struct ClusterLevels {
    int nd;                        // distributed levels
    int n0[MG_CL_MAX_LEVELS], n1[MG_CL_MAX_LEVELS], n2[MG_CL_MAX_LEVELS], P[MG_CL_MAX_LEVELS];
    FastDiv dh[MG_CL_MAX_LEVELS];  // n0 / 2
    FastDiv d0[MG_CL_MAX_LEVELS];  // n0
    FastDiv d1[MG_CL_MAX_LEVELS];  // n1
    float kh2f[MG_CL_MAX_LEVELS], invf[MG_CL_MAX_LEVELS];  // as in TailLevels
    double kh2d[MG_CL_MAX_LEVELS], invd[MG_CL_MAX_LEVELS];
    int uoff[MG_CL_MAX_LEVELS];    // u slab of level l in every CTA's shared memory (elements)
    int foff[MG_CL_MAX_LEVELS];    // f slab (levels >= 1)
    int toff;                      // tail region (CTA 0)
    TailLevels tail;               // offsets relative to toff
};

template <typename T>
__global__ void __launch_bounds__(1024) k_mg_cluster(const __grid_constant__ ClusterLevels cl, T* __restrict__ ug,
                                                     const T* __restrict__ fg,
                                                     T sigma, int zero_start, int pre, int post, int sweeps) {
    pdl_start();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sm = reinterpret_cast<T*>(smem_raw);
    __shared__ double red[32];
    cg::cluster_group cluster = cg::this_cluster();
    const int r = (int)cluster.block_rank();
    const int cmp = blockIdx.x / MG_CL;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int plane0 = cl.n0[0] * cl.n1[0];
    const long long ncell0 = (long long)plane0 * cl.n2[0];
    ug += cmp * ncell0;
    fg += cmp * ncell0;
    T* tailbase = sm + cl.toff;

    // pointer to plane k (any, wrapped) of the u (or f) slabs of distributed level l
    auto dplane = [&](int l, int off, int k) -> T* {
        const int n2 = cl.n2[l], P = cl.P[l];
        k = k < 0 ? k + n2 : (k >= n2 ? k - n2 : k);
        const int owner = k / P;
        return cluster.map_shared_rank(sm + off, owner) + (k - owner * P) * (cl.n0[l] * cl.n1[l]);
    };
    // red-black half sweep of distributed level l
    auto dhalf = [&](int l, int color, int zero) {
        const int n0 = cl.n0[l], n1 = cl.n1[l], P = cl.P[l], hn0 = n0 >> 1;
        const int plane = n0 * n1;
        T* u = sm + cl.uoff[l];
        const T* ub = dplane(l, cl.uoff[l], r * P - 1);
        const T* ua = dplane(l, cl.uoff[l], r * P + P);
        const T* f = l == 0 ? fg + (long long)r * P * plane : sm + cl.foff[l];
        const T kh2 = lev_kh2<T>(cl, l);
        const T inv = lev_inv<T>(cl, l);
        const int np = P * n1 * hn0;
        for (int t = tid; t < np; t += nt) {
            const int q = fdiv(t, cl.dh[l]);
            const int ih = t - q * hn0;
            const int kl = fdiv(q, cl.d1[l]);
            const int j = q - kl * n1;
            const int i = 2 * ih + ((j + r * P + kl + color) & 1);
            const int c = i + n0 * j;
            T* pc = u + kl * plane;
            const T* pm = kl == 0 ? ub : pc - plane;
            const T* pp = kl == P - 1 ? ua : pc + plane;
            const int xp = (i == n0 - 1) ? 1 - n0 : 1;
            const int xm = (i == 0) ? n0 - 1 : -1;
            const int yp = (j == n1 - 1) ? (1 - n1) * n0 : n0;
            const int ym = (j == 0) ? (n1 - 1) * n0 : -n0;
            T nb = T(0);
            if (!zero) {
                nb = pc[c + xp] + pc[c + xm] + pc[c + yp] + pc[c + ym];
                nb += pp[c] + pm[c];
            }
            pc[c] = (f[kl * plane + c] + kh2 * nb) * inv;
        }
        cluster.sync();
    };
    // residual of distributed level l at its cell (i, j, k) (k global)
    auto dresid = [&](int l, int i, int j, int k, T kh2) -> T {
        const int n0 = cl.n0[l], n1 = cl.n1[l];
        const T* pc = dplane(l, cl.uoff[l], k);
        const T* pm = dplane(l, cl.uoff[l], k - 1);
        const T* pp = dplane(l, cl.uoff[l], k + 1);
        const T* fp = l == 0 ? fg + (long long)k * n0 * n1 : dplane(l, cl.foff[l], k);
        const int c = i + n0 * j;
        const int xp = (i == n0 - 1) ? 1 - n0 : 1;
        const int xm = (i == 0) ? n0 - 1 : -1;
        const int yp = (j == n1 - 1) ? (1 - n1) * n0 : n0;
        const int ym = (j == 0) ? (n1 - 1) * n0 : -n0;
        const T uc = pc[c];
        T nbs = pc[c + xp] + pc[c + xm] + pc[c + yp] + pc[c + ym];
        nbs += pp[c] + pm[c];
        return fp[c] - (sigma * uc - kh2 * (nbs - T(6) * uc));
    };
    // f of level l+1 = the averaged residual of distributed level l, for the
    // coarse planes K whose first fine plane 2K this CTA owns
    auto drestrict = [&](int l) {
        const int n0c = cl.n0[l] >> 1, n1c = cl.n1[l] >> 1;
        const int planec = n0c * n1c;
        const int P = cl.P[l];
        const int K0 = (r * P + 1) >> 1, K1 = (r * P + P + 1) >> 1;  // 2K in [rP, rP + P)
        const bool coarse_dist = l + 1 < cl.nd;
        const FastDiv dc0 = coarse_dist ? cl.d0[l + 1] : cl.tail.d0[0];
        const int np = (K1 - K0) * planec;
        const T kh2 = lev_kh2<T>(cl, l);
        for (int t = tid; t < np; t += nt) {
            const int q = fdiv(t, dc0);
            const int I = t - q * n0c;
            const int kk = q / n1c;
            const int J = q - kk * n1c;
            const int K = K0 + kk;
            T acc = T(0);
#pragma unroll
            for (int c = 0; c < 8; ++c)
                acc += dresid(l, 2 * I + (c & 1), 2 * J + ((c >> 1) & 1), 2 * K + ((c >> 2) & 1), kh2);
            T* fcp = coarse_dist ? dplane(l + 1, cl.foff[l + 1], K)
                                 : cluster.map_shared_rank(tailbase + cl.tail.foff[0], 0) + K * planec;
            fcp[I + n0c * J] = acc * (T(1) / T(8));
        }
        cluster.sync();
    };
    // u of distributed level l += prolongation of level l+1's u (own planes)
    auto dprolong = [&](int l) {
        const int n0 = cl.n0[l], n1 = cl.n1[l], P = cl.P[l];
        const int plane = n0 * n1;
        const int n0c = n0 >> 1, n1c = n1 >> 1, n2c = cl.n2[l] >> 1;
        const bool coarse_dist = l + 1 < cl.nd;
        T* u = sm + cl.uoff[l];
        const int np = P * plane;
        const T w[2] = {T(0.75), T(0.25)};
        for (int t = tid; t < np; t += nt) {
            const int q = fdiv(t, cl.d0[l]);
            const int i = t - q * n0;
            const int kl = fdiv(q, cl.d1[l]);
            const int j = q - kl * n1;
            const int k = r * P + kl;
            int I[2], Jc[2], Kc[2];
            I[0] = i >> 1;
            I[1] = (i & 1) ? (I[0] + 1 == n0c ? 0 : I[0] + 1) : (I[0] == 0 ? n0c - 1 : I[0] - 1);
            Jc[0] = j >> 1;
            Jc[1] = (j & 1) ? (Jc[0] + 1 == n1c ? 0 : Jc[0] + 1) : (Jc[0] == 0 ? n1c - 1 : Jc[0] - 1);
            Kc[0] = k >> 1;
            Kc[1] = (k & 1) ? (Kc[0] + 1 == n2c ? 0 : Kc[0] + 1) : (Kc[0] == 0 ? n2c - 1 : Kc[0] - 1);
            const T* cp[2];
#pragma unroll
            for (int e = 0; e < 2; ++e)
                cp[e] = coarse_dist ? dplane(l + 1, cl.uoff[l + 1], Kc[e])
                                    : cluster.map_shared_rank(tailbase + cl.tail.uoff[0], 0) + Kc[e] * (n0c * n1c);
            T acc = T(0);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int a = c & 1, b = (c >> 1) & 1, e = (c >> 2) & 1;
                const T ww = w[a] * w[b] * w[e];
                acc += ww * cp[e][I[a] + n0c * Jc[b]];
            }
            u[t] += acc;
        }
        cluster.sync();
    };

    // the top level's u slab from global memory (or zero)
    {
        T* u0 = sm + cl.uoff[0];
        const int n = cl.P[0] * plane0;
        const T* src = ug + (long long)r * n;
        for (int c = tid; c < n; c += nt) u0[c] = zero_start ? T(0) : src[c];
    }
    cluster.sync();
    const int nd = cl.nd;
    for (int l = 0; l < nd; ++l) {
        const int zs = (l > 0) || zero_start;
        if (pre == 0 && zs) {
            T* u = sm + cl.uoff[l];
            for (int c = tid; c < cl.P[l] * cl.n0[l] * cl.n1[l]; c += nt) u[c] = T(0);
            cluster.sync();
        }
        for (int it = 0; it < pre; ++it) {
            dhalf(l, 0, zs && it == 0);
            dhalf(l, 1, 0);
        }
        drestrict(l);
    }
    if (r == 0) tail_solve<3, false, T>(cl.tail, tailbase, 0, sigma, 1, pre, post, sweeps, red);
    cluster.sync();
    for (int l = nd - 1; l >= 0; --l) {
        dprolong(l);
        for (int it = 0; it < post; ++it) {
            dhalf(l, 1, 0);
            dhalf(l, 0, 0);
        }
    }
    {
        const T* u0 = sm + cl.uoff[0];
        const int n = cl.P[0] * plane0;
        T* dst = ug + (long long)r * n;
        for (int c = tid; c < n; c += nt) dst[c] = u0[c];
    }
}

// q = -D y - hd ; qr = rhs_scale * q
template <int D, bool W, typename T>
__global__ void __launch_bounds__(256) k_ps_div(const T* __restrict__ y, const T* __restrict__ hd,
                                                T* __restrict__ qr, T rhs_scale, T* __restrict__ q, Geo g, T ih) {
    pdl_start();
    int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
    if (i >= g.n0 || j >= g.n1) return;
    Nbr n = neighbours<D>(g, i, j, k);
    const int pp[3] = {n.xp, n.yp, n.zp};
    const int id[3] = {i, j, k};
    const int ns[3] = {g.n0, g.n1, g.n2};
    T div = T(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const T* u = y + a * g.ncell;
        if (!W) {
            div += u[n.c + pp[a]] - u[n.c];
        } else {
            const bool wa = (g.wall >> a) & 1;
            T hi = (wa && id[a] == ns[a] - 1) ? T(0) : u[n.c + pp[a]];
            T lo = (wa && id[a] == 0) ? T(0) : u[n.c];
            div += hi - lo;
        }
    }
    T qq = -div * ih - hd[n.c];
    q[n.c] = qq;
    qr[n.c] = rhs_scale * qq;
}

// z_v^a = y^a + h^2 (G phi)^a = y^a + h (phi_c - phi_{c-e_a}) (wall faces:
// no gradient) ; z_p = c_q q + c_phi phi
template <int D, bool W, typename T>
__global__ void __launch_bounds__(256) k_ps_finish(const T* __restrict__ y, const T* __restrict__ phi,
                                                   const T* __restrict__ q, T* __restrict__ z, Geo g, T h, T c_q,
                                                   T c_phi) {
    pdl_start();
    int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
    if (i >= g.n0 || j >= g.n1) return;
    Nbr n = neighbours<D>(g, i, j, k);
    const int pm[3] = {n.xm, n.ym, n.zm};
    const int id[3] = {i, j, k};
    T pc = phi[n.c];
#pragma unroll
    for (int a = 0; a < D; ++a) {
        if (W && ((g.wall >> a) & 1) && id[a] == 0)
            z[a * g.ncell + n.c] = y[a * g.ncell + n.c];
        else
            z[a * g.ncell + n.c] = y[a * g.ncell + n.c] + h * (pc - phi[n.c + pm[a]]);
    }
    z[D * g.ncell + n.c] = c_q * q[n.c] + c_phi * pc;
}

// boundary data of one wall into the right-hand side (one thread per face point)
__global__ void k_wall_lift(Geo g, int a, int side, const double* __restrict__ data, double* __restrict__ b,
                            double kh2, double ih) {
    const int ns[3] = {g.n0, g.n1, g.n2};
    const long long nf = g.ncell / ns[a];
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= nf) return;
    int id[3] = {0, 0, 0};
    long long r = t;
    for (int e = 0; e < g.d; ++e) {
        if (e == a) continue;
        id[e] = (int)(r % ns[e]);
        r /= ns[e];
    }
    const long long st[3] = {1, ns[0], (long long)ns[0] * ns[1]};
    auto cell = [&](int xa) {
        long long c = 0;
        for (int e = 0; e < g.d; ++e) c += (long long)(e == a ? xa : id[e]) * st[e];
        return c;
    };
    const int n = ns[a];
    double* bp = b + (long long)g.d * g.ncell;
    for (int c = 0; c < g.d; ++c) {
        const double val = data[c * nf + t];
        double* bc = b + (long long)c * g.ncell;
        if (c == a) {
            if (side == 0) {
                bc[cell(0)] = val;         // the wall face: v = wall value
                bc[cell(1)] += kh2 * val;  // its neighbour face
                bp[cell(0)] -= ih * val;   // inflow through the low face of cell 0
            } else {
                bc[cell(n - 1)] += kh2 * val;
                bp[cell(n - 1)] += ih * val;
            }
        } else {
            // the cell next to the wall: ghost = 2 u_wall - u; a wall-face
            // row of component c keeps its own equation
            if (((g.wall >> c) & 1) && id[c] == 0) continue;
            bc[cell(side ? n - 1 : 0)] += 2.0 * kh2 * val;
        }
    }
}

// the stored low-wall faces of the normal component set to the wall value
__global__ void k_wall_set(Geo g, int a, const double* __restrict__ data, double* __restrict__ x) {
    const int ns[3] = {g.n0, g.n1, g.n2};
    const long long nf = g.ncell / ns[a];
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= nf) return;
    long long r = t, c = 0, st = 1;
    for (int e = 0; e < g.d; ++e) {
        if (e != a) {
            c += (r % ns[e]) * st;
            r /= ns[e];
        }
        st *= ns[e];
    }
    x[(long long)a * g.ncell + c] = data[(long long)a * nf + t];
}

}  // namespace

void wall_set_faces(const Geo& g, int a, const double* data, double* x, cudaStream_t s) {
    const int ns[3] = {g.n0, g.n1, g.n2};
    long long nf = g.ncell / ns[a];
    ProfScope ps(KID_SMALL, s, 0.0);
    k_wall_set<<<grid_1d(nf, 128), 128, 0, s>>>(g, a, data, x);
    IBR_CHECK_LAUNCH();
}

template <typename T>
void stokes_apply(const Geo& g, const T* x, T* y, double sigma, double eta, const double* shift_dev,
                  cudaStream_t s) {
    T kh2 = (T)(eta / (g.h * g.h));
    T ih = (T)(1.0 / g.h);
    dim3 grid((g.n0 + BX - 1) / BX, (g.n1 + BY - 1) / BY, g.n2), blk(BX, BY);
    ProfScope ps(KID_STOKES, s, 2.0 * (g.d + 1) * g.ncell * sizeof(T));
    const bool w = g.wall != 0;
    if (g.d == 3) {
        if (w)
            launch_k(k_stokes<3, true, T>, grid, blk, 0, s, x, y, g, (T)sigma, kh2, ih, shift_dev);
        else
            launch_k(k_stokes<3, false, T>, grid, blk, 0, s, x, y, g, (T)sigma, kh2, ih, shift_dev);
    } else {
        if (w)
            launch_k(k_stokes<2, true, T>, grid, blk, 0, s, x, y, g, (T)sigma, kh2, ih, shift_dev);
        else
            launch_k(k_stokes<2, false, T>, grid, blk, 0, s, x, y, g, (T)sigma, kh2, ih, shift_dev);
    }
    IBR_CHECK_LAUNCH();
}

// Tile autotuner of the periodic 3-D column smoother: per level shape (n0,
// n1, n2, C, element size) the block height by (of 32 x by threads) and the
// column length kz with the shortest measured half sweep.  Tuning runs once
// per shape and process, on scratch arrays (the result does not depend on
// the tile), outside stream capture (from the multigrid set-up); until a
// shape is tuned, or with IBR_TUNE=0, the fixed heuristic tile is used.
struct ColTile {
    int by, kz;
};
std::mutex g_tile_mu;
std::map<std::array<long long, 5>, ColTile> g_tiles;

ColTile col_tile_heuristic(const Geo& g, int C) {
    // columns of kz cells; kz shrinks on small levels to keep ~1.5e5 threads busy
    const long long cells = (long long)(g.n0 >> 1) * g.n1 * g.n2 * C;
    return ColTile{BY, (int)std::min<long long>(8, std::max<long long>(1, cells / 150000))};
}

ColTile col_tile(const Geo& g, int C, size_t esz) {
    std::lock_guard<std::mutex> lk(g_tile_mu);
    auto it = g_tiles.find({g.n0, g.n1, g.n2, C, (long long)esz});
    return it != g_tiles.end() ? it->second : col_tile_heuristic(g, C);
}

template <typename T>
void launch_col(const Geo& g, T* u, const T* f, int C, ColTile t, T kh2, T inv, int color, int zi, cudaStream_t s) {
    const int nkb = (g.n2 + t.kz - 1) / t.kz;
    dim3 gc(((g.n0 >> 1) + 31) / 32, (g.n1 + t.by - 1) / t.by, nkb * C), blk(32, t.by);
    launch_k(k_rbgs_col<T>, gc, blk, 0, s, u, f, g, nkb, t.kz, kh2, inv, color, zi);
}

template <typename T>
void mg_tune_smoother(const Geo& g, int C, cudaStream_t s) {
    if (g.d != 3 || g.wall) return;
    const long long cells = (long long)(g.n0 >> 1) * g.n1 * g.n2 * C;
    if (cells < (1LL << 17)) return;  // small levels: latency-bound, the heuristic is fine
    static const bool off = [] {
        const char* e = std::getenv("IBR_TUNE");
        return e && e[0] == '0';
    }();
    if (off) return;
    const std::array<long long, 5> key = {g.n0, g.n1, g.n2, C, (long long)sizeof(T)};
    {
        std::lock_guard<std::mutex> lk(g_tile_mu);
        if (g_tiles.count(key)) return;
    }
    cudaStreamCaptureStatus cs;
    IBR_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) return;
    const size_t n = (size_t)C * g.ncell;
    T *u = nullptr, *f = nullptr;
    IBR_CUDA_TRY(cudaMallocAsync(&u, n * sizeof(T), s));
    IBR_CUDA_TRY(cudaMallocAsync(&f, n * sizeof(T), s));
    IBR_CUDA_TRY(cudaMemsetAsync(u, 0, n * sizeof(T), s));
    IBR_CUDA_TRY(cudaMemsetAsync(f, 0, n * sizeof(T), s));
    cudaEvent_t e0, e1;
    IBR_CUDA_TRY(cudaEventCreate(&e0));
    IBR_CUDA_TRY(cudaEventCreate(&e1));
    const T kh2 = (T)1, inv = (T)(1.0 / 6.0);
    ColTile best = col_tile_heuristic(g, C);
    float best_ms = 1e30f;
    const int bys[] = {4, 8};  // 32 x by threads within the kernel's launch bound of 256
    const int kzs[] = {2, 4, 6, 8, 11, 16, 22, 32};
    for (int by : bys)
        for (int kz : kzs) {
            if (kz > g.n2) continue;
            const ColTile t{by, kz};
            for (int r = 0; r < 2; ++r) launch_col<T>(g, u, f, C, t, kh2, inv, r & 1, 0, s);
            IBR_CUDA_TRY(cudaEventRecord(e0, s));
            for (int r = 0; r < 6; ++r) launch_col<T>(g, u, f, C, t, kh2, inv, r & 1, 0, s);
            IBR_CUDA_TRY(cudaEventRecord(e1, s));
            IBR_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            IBR_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best_ms) {
                best_ms = ms;
                best = t;
            }
        }
    IBR_CUDA_TRY(cudaGetLastError());
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    IBR_CUDA_TRY(cudaFreeAsync(u, s));
    IBR_CUDA_TRY(cudaFreeAsync(f, s));
    std::lock_guard<std::mutex> lk(g_tile_mu);
    g_tiles[key] = best;
}

bool tuned_tile(int idx, int* out7) {
    std::lock_guard<std::mutex> lk(g_tile_mu);
    if (idx < 0 || idx >= (int)g_tiles.size()) return false;
    auto it = g_tiles.begin();
    std::advance(it, idx);
    for (int q = 0; q < 5; ++q) out7[q] = (int)it->first[q];
    out7[5] = it->second.by;
    out7[6] = it->second.kz;
    return true;
}

template <typename T>
void mg_smooth(const Geo& g, T* u, const T* f, int C, int fld0, double sigma, double kappa, int color,
               bool zero_init, cudaStream_t s) {
    T kh2 = (T)(kappa / (g.h * g.h));
    dim3 grid(((g.n0 >> 1) + BX - 1) / BX, (g.n1 + BY - 1) / BY, g.n2 * C), blk(BX, BY);
    // half sweep: read the other colour and f of this colour, write this colour
    ProfScope ps(KID_RBGS, s, (zero_init ? 1.0 : 1.5) * C * g.ncell * sizeof(T));
    const int zi = zero_init ? 1 : 0;
    const T sg = (T)sigma;
    if (g.d == 3) {
        T inv = rbgs_inv_diag<3, T>(sg, kh2);
        if (g.wall) {
            launch_k(k_rbgs<3, true, T>, grid, blk, 0, s, u, f, g, fld0, sg, kh2, inv, color, zi);
        } else {
            launch_col<T>(g, u, f, C, col_tile(g, C, sizeof(T)), kh2, inv, color, zi, s);
        }
    } else {
        T inv = rbgs_inv_diag<2, T>(sg, kh2);
        if (g.wall)
            launch_k(k_rbgs<2, true, T>, grid, blk, 0, s, u, f, g, fld0, sg, kh2, inv, color, zi);
        else
            launch_k(k_rbgs<2, false, T>, grid, blk, 0, s, u, f, g, fld0, sg, kh2, inv, color, zi);
    }
    IBR_CHECK_LAUNCH();
}

template <typename T>
void mg_residual_restrict(const Geo& gf, const Geo& gc, const T* u, const T* f, T* fc, int C, int fld0,
                          double sigma, double kappa, cudaStream_t s) {
    T kh2 = (T)(kappa / (gf.h * gf.h));
    dim3 grid((gc.n0 + BX - 1) / BX, (gc.n1 + BY - 1) / BY, gc.n2 * C), blk(BX, BY);
    ProfScope ps(KID_RESTRICT, s, (2.0 * gf.ncell + gc.ncell) * C * sizeof(T));
    if (gf.d == 3) {
        if (gf.wall)
            launch_k(k_resid_restrict<3, true, T>, grid, blk, 0, s, u, f, fc, gf, gc, fld0, (T)sigma, kh2);
        else
            launch_k(k_resid_restrict<3, false, T>, grid, blk, 0, s, u, f, fc, gf, gc, fld0, (T)sigma, kh2);
    } else {
        if (gf.wall)
            launch_k(k_resid_restrict<2, true, T>, grid, blk, 0, s, u, f, fc, gf, gc, fld0, (T)sigma, kh2);
        else
            launch_k(k_resid_restrict<2, false, T>, grid, blk, 0, s, u, f, fc, gf, gc, fld0, (T)sigma, kh2);
    }
    IBR_CHECK_LAUNCH();
}

template <typename T>
void mg_prolong_correct(const Geo& gf, const Geo& gc, T* u, const T* uc, int C, int fld0, cudaStream_t s) {
    dim3 grid((gf.n0 + BX - 1) / BX, (gf.n1 + BY - 1) / BY, gf.n2 * C), blk(BX, BY);
    ProfScope ps(KID_PROLONG, s, (2.0 * gf.ncell + gc.ncell) * C * sizeof(T));
    if (gf.d == 3) {
        if (gf.wall)
            launch_k(k_prolong<3, true, T>, grid, blk, 0, s, u, uc, gf, gc, fld0);
        else
            launch_k(k_prolong<3, false, T>, grid, blk, 0, s, u, uc, gf, gc, fld0);
    } else {
        if (gf.wall)
            launch_k(k_prolong<2, true, T>, grid, blk, 0, s, u, uc, gf, gc, fld0);
        else
            launch_k(k_prolong<2, false, T>, grid, blk, 0, s, u, uc, gf, gc, fld0);
    }
    IBR_CHECK_LAUNCH();
}

template <typename T>
void mg_coarse_solve(const Geo& g, T* u, const T* f, int C, int fld0, double sigma, double kappa, int sweeps,
                     cudaStream_t s) {
    T kh2 = (T)(kappa / (g.h * g.h));
    size_t sm = 2 * (size_t)g.ncell * sizeof(T);
    int nt = g.ncell >= 1024 ? 1024 : (int)((g.ncell + 31) / 32 * 32);
    ProfScope ps(KID_COARSE, s, 2.0 * C * g.ncell * sizeof(T));
    const FastDiv d0 = make_fastdiv(g.n0), d1 = make_fastdiv(g.n1);
    const T inv = g.d == 3 ? rbgs_inv_diag<3, T>((T)sigma, kh2) : rbgs_inv_diag<2, T>((T)sigma, kh2);
    if (g.d == 3) {
        if (g.wall)
            k_coarse<3, true, T><<<C, nt, sm, s>>>(u, f, g, fld0, (T)sigma, kh2, inv, sweeps, d0, d1);
        else
            k_coarse<3, false, T><<<C, nt, sm, s>>>(u, f, g, fld0, (T)sigma, kh2, inv, sweeps, d0, d1);
    } else {
        if (g.wall)
            k_coarse<2, true, T><<<C, nt, sm, s>>>(u, f, g, fld0, (T)sigma, kh2, inv, sweeps, d0, d1);
        else
            k_coarse<2, false, T><<<C, nt, sm, s>>>(u, f, g, fld0, (T)sigma, kh2, inv, sweeps, d0, d1);
    }
    IBR_CHECK_LAUNCH();
}

// the tail kernels' shared-memory limit, raised once per device (function
// attributes belong to the device that is current when they are set)
template <typename T>
void mg_set_attributes() {
    static PerDeviceOnce once;
    once.run([] {
        const int sm = (int)MG_TAIL_MAX_SMEM;
        IBR_CUDA_TRY(cudaFuncSetAttribute(k_mg_tail<3, false, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
        IBR_CUDA_TRY(cudaFuncSetAttribute(k_mg_tail<2, false, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
        IBR_CUDA_TRY(cudaFuncSetAttribute(k_mg_tail<3, true, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
        IBR_CUDA_TRY(cudaFuncSetAttribute(k_mg_tail<2, true, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
    });
}

// shared memory of the tail kernel for levels [l0, L)
template <typename T>
static size_t tail_smem(const Geo* lev, int l0, int L) {
    size_t n = 0;
    for (int l = l0; l < L; ++l) n += 2 * (size_t)lev[l].ncell;
    return n * sizeof(T);
}

// tail levels [lt, L) in a TailLevels (offsets from 0, in elements)
// kappa h^-2 and 1 / (sigma + 2D kappa h^-2) of a level, in float and double
// (the same expressions as the per-level launches)
template <typename L>
void level_coefs(L& x, int q, const Geo& g, double sigma, double kappa) {
    x.kh2f[q] = (float)(kappa / (g.h * g.h));
    x.kh2d[q] = kappa / (g.h * g.h);
    x.invf[q] = g.d == 3 ? rbgs_inv_diag<3, float>((float)sigma, x.kh2f[q]) : rbgs_inv_diag<2, float>((float)sigma, x.kh2f[q]);
    x.invd[q] = g.d == 3 ? rbgs_inv_diag<3, double>(sigma, x.kh2d[q]) : rbgs_inv_diag<2, double>(sigma, x.kh2d[q]);
}

template <typename T>
TailLevels make_tail(const Geo* lev, int lt, int L, double sigma, double kappa) {
    TailLevels tl;
    tl.nl = L - lt;
    int off = 0;
    for (int q = 0; q < tl.nl; ++q) {
        tl.g[q] = lev[lt + q];
        tl.uoff[q] = off;
        off += (int)lev[lt + q].ncell;
        tl.foff[q] = off;
        off += (int)lev[lt + q].ncell;
        tl.dh[q] = make_fastdiv(lev[lt + q].n0 / 2);
        tl.d0[q] = make_fastdiv(lev[lt + q].n0);
        tl.d1[q] = make_fastdiv(lev[lt + q].n1);
        level_coefs(tl, q, lev[lt + q], sigma, kappa);
    }
    return tl;
}

// the first tail level: the longest suffix of levels with <= MG_TAIL_MAX_CELLS
// cells each that fits in shared memory (the coarsest level always does)
template <typename T>
int tail_start(const Geo* lev, int L) {
    int lt = L - 1;
    while (lt - 1 >= 0 && L - (lt - 1) <= MG_TAIL_MAX_LEVELS && lev[lt - 1].ncell <= MG_TAIL_MAX_CELLS &&
           tail_smem<T>(lev, lt - 1, L) <= MG_TAIL_MAX_SMEM)
        --lt;
    return lt;
}

// Cluster plan of a periodic 3-D hierarchy: levels [top, top + nd) distributed
// over the MG_CL CTAs of a cluster (n2 a multiple of MG_CL), the tail [top +
// nd, L) in CTA 0; top as fine as shared memory allows.  false: no such plan.
constexpr size_t MG_CL_SMEM = 200 * 1024;
// want: the top level to use (-1: the finest feasible level with at most
// MG_CL_DEFAULT_TOP_CELLS cells: larger levels keep more of the GPU busy with
// one launch per sweep than one 8-CTA cluster per field can)
constexpr long long MG_CL_DEFAULT_TOP_CELLS = 32768;
template <typename T>
bool cluster_plan(const Geo* lev, int L, double sigma, double kappa, int want, int& top, ClusterLevels& cl) {
    if (lev[0].d != 3 || lev[0].wall) return false;
    const int lt = tail_start<T>(lev, L);
    if (lt < 1) return false;
    // distributed levels must be above the tail and split evenly in z
    for (int t = 0; t < lt; ++t) {
        if (want >= 0 ? t != want : lev[t].ncell > MG_CL_DEFAULT_TOP_CELLS) continue;
        bool ok = lt - t <= MG_CL_MAX_LEVELS;
        size_t bytes = tail_smem<T>(lev, lt, L);
        for (int l = t; l < lt && ok; ++l) {
            const Geo& g = lev[l];
            if (g.n2 % MG_CL != 0 || g.n0 % 2 != 0) ok = false;
            const size_t slab = (size_t)(g.n2 / MG_CL) * g.n0 * g.n1 * sizeof(T);
            bytes += l == t ? slab : 2 * slab;
        }
        if (!ok || bytes + 64 > MG_CL_SMEM) continue;
        top = t;
        cl.nd = lt - t;
        int off = 0;
        for (int q = 0; q < cl.nd; ++q) {
            const Geo& g = lev[t + q];
            cl.n0[q] = g.n0;
            cl.n1[q] = g.n1;
            cl.n2[q] = g.n2;
            cl.P[q] = g.n2 / MG_CL;
            level_coefs(cl, q, g, sigma, kappa);
            cl.dh[q] = make_fastdiv(g.n0 / 2);
            cl.d0[q] = make_fastdiv(g.n0);
            cl.d1[q] = make_fastdiv(g.n1);
            const int slab = cl.P[q] * g.n0 * g.n1;
            cl.uoff[q] = off;
            off += slab;
            cl.foff[q] = q == 0 ? -1 : off;
            if (q > 0) off += slab;
        }
        cl.toff = (off + 3) & ~3;
        cl.tail = make_tail<T>(lev, lt, L, sigma, kappa);
        return true;
    }
    return false;
}

// whether this device runs MG_CL-CTA clusters of k_mg_cluster with MG_CL_SMEM
// bytes of shared memory (checked once per device; IBR_MG_CLUSTER=0 in the
// environment: never)
template <typename T>
bool cluster_ok() {
    static const bool off = [] {
        const char* e = std::getenv("IBR_MG_CLUSTER");
        return e && e[0] == '0';
    }();
    if (off) return false;
    static std::mutex mu;
    static int state[128] = {0};  // 0 unknown, 1 yes, 2 no
    int dev = 0;
    IBR_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) return false;
    std::lock_guard<std::mutex> lk(mu);
    if (state[dev] == 0) {
        state[dev] = 2;
        if (cudaFuncSetAttribute(k_mg_cluster<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MG_CL_SMEM) ==
            cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = MG_CL;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.gridDim = dim3(MG_CL, 1, 1);
            cfg.blockDim = dim3(1024, 1, 1);
            cfg.dynamicSmemBytes = MG_CL_SMEM;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int nc = 0;
            if (cudaOccupancyMaxActiveClusters(&nc, k_mg_cluster<T>, &cfg) == cudaSuccess && nc >= 1) state[dev] = 1;
        }
        cudaGetLastError();  // a refused query leaves no error behind
    }
    return state[dev] == 1;
}

// The V-cycle schedule autotuner's choice per hierarchy (finest level shape,
// levels, stacked fields, element size): the level the cluster kernel starts
// at, or -2 for none (per-level kernels and the one-CTA tail).
std::mutex g_cl_mu;
std::map<std::array<long long, 6>, int> g_cl_top;

std::array<long long, 6> cl_key(const Geo* lev, int L, int C, size_t esz) {
    return {lev[0].n0, lev[0].n1, lev[0].n2, L, C, (long long)esz};
}

// IBR_MG_CLUSTER_LEVEL=<level> in the environment: the cluster kernel from
// that level whenever feasible (measurement and tests); -1 when unset
int cluster_forced() {
    static const int lv = [] {
        const char* e = std::getenv("IBR_MG_CLUSTER_LEVEL");
        return (e && e[0] >= '0' && e[0] <= '9') ? std::atoi(e) : -1;
    }();
    return lv;
}

int cluster_choice(const Geo* lev, int L, int C, size_t esz) {
    if (cluster_forced() >= 0) return cluster_forced();
    std::lock_guard<std::mutex> lk(g_cl_mu);
    auto it = g_cl_top.find(cl_key(lev, L, C, esz));
    return it == g_cl_top.end() ? -1 : it->second;
}

// whether the finest level of this V-cycle runs in red-black split layout
// (IBR_MG_SPLIT=0 in the environment: never)
template <typename T>
bool rb_split_ok(const Geo& g, const T* F0, const T* U0, const T* rb_u, const T* rb_f, bool zero_start, int pre,
                 int post) {
    static const bool off = [] {
        const char* e = std::getenv("IBR_MG_SPLIT");
        return e && e[0] == '0';
    }();
    const uintptr_t al = (uintptr_t)(RB_V * sizeof(T) * 2);
    return !off && rb_u && rb_f && g.d == 3 && !g.wall && g.n0 % (2 * RB_V) == 0 && zero_start && pre >= 1 &&
           post >= 1 &&
           (((uintptr_t)F0 | (uintptr_t)U0 | (uintptr_t)rb_u | (uintptr_t)rb_f) % al) == 0;
}

// (the caller's profile scope covers the launch)
template <typename T>
void rb_launch_half(const Geo& g, int C, T* us, const T* fs, T kh2, T inv, int color, T* unat, cudaStream_t s) {
    const int nth = (int)((long long)C * g.ncell / (2 * RB_V));
    const int hq = g.n0 / (2 * RB_V);
    launch_k(k_rb_half<T>, dim3(grid_1d(nth, 256)), dim3(256), 0, s, us, fs, g.n0, g.n1, g.n2, nth,
             make_fastdiv(hq), make_fastdiv(g.n1), make_fastdiv(g.n2), kh2, inv, color, unat);
    IBR_CHECK_LAUNCH();
}

template <typename T>
void mg_vcycle(const Geo* lev, int L, T* const* U, T* const* Fw, const T* F0, int C, int fld0, double sigma,
               double kappa, bool zero_start, int pre, int post, int coarse_sweeps, cudaStream_t s, T* rb_u,
               T* rb_f, T* rb_u1, T* rb_f1) {
    auto Fl = [&](int l) -> const T* { return l == 0 ? F0 : Fw[l]; };
    // periodic 3-D: the finest level and the next in red-black split layout
    // (conversions folded into the first and last half sweeps of each)
    T* rbu[2] = {rb_u, rb_u1};
    T* rbf[2] = {rb_f, rb_f1};
    bool split_l[2];
    for (int l = 0; l < 2; ++l)
        split_l[l] = L > l + 1 && (long long)C * lev[l].ncell < (1LL << 31) &&
                     rb_split_ok<T>(lev[l], Fl(l), U[l], rbu[l], rbf[l], l > 0 || zero_start, pre, post);
    auto split = [&](int l) { return l < 2 && split_l[l]; };
    // periodic 3-D: the coarse levels on one thread-block cluster per field
    ClusterLevels cl;
    int top = 0;
    const int want = cluster_choice(lev, L, C, sizeof(T));
    const bool use_cluster =
        want != -2 && cluster_plan<T>(lev, L, sigma, kappa, want, top, cl) && cluster_ok<T>();
    const int lt = use_cluster ? top : tail_start<T>(lev, L);
    for (int l = 0; l < lt; ++l) {
        if (split(l)) {
            const Geo& g = lev[l];
            T* ru = rbu[l];
            T* rf = rbf[l];
            const T rb_kh2 = (T)(kappa / (g.h * g.h));
            const T rb_inv = rbgs_inv_diag<3, T>((T)sigma, rb_kh2);
            const int nth = (int)((long long)C * g.ncell / (2 * RB_V));
            {
                // the pre-smoothing half sweeps, timed as one back-to-back sequence
                ProfScope ps(KID_RBGS, s, (1.0 + 3.0 * pre) * C * g.ncell * sizeof(T), 0.0, 2 * pre);
                launch_k(k_rb_first<T>, dim3(grid_1d(nth, 256)), dim3(256), 0, s, Fl(l), rf, ru, g.n0, g.n1, g.n2,
                         nth, make_fastdiv(g.n0 / (2 * RB_V)), make_fastdiv(g.n1), make_fastdiv(g.n2), rb_inv);
                IBR_CHECK_LAUNCH();
                rb_launch_half<T>(g, C, ru, rf, rb_kh2, rb_inv, 1, (T*)nullptr, s);
                for (int it = 1; it < pre; ++it) {
                    rb_launch_half<T>(g, C, ru, rf, rb_kh2, rb_inv, 0, (T*)nullptr, s);
                    rb_launch_half<T>(g, C, ru, rf, rb_kh2, rb_inv, 1, (T*)nullptr, s);
                }
            }
            const Geo& gc = lev[l + 1];
            const long long ncc = gc.ncell * C;
            ProfScope ps(KID_RESTRICT, s, (2.0 * g.ncell + gc.ncell) * C * sizeof(T));
            launch_k(k_rb_restrict<T>, dim3(grid_1d(ncc, 256)), dim3(256), 0, s, (const T*)ru, (const T*)rf,
                     Fw[l + 1], g.n0, g.n1, g.n2, C, (T)sigma, rb_kh2, make_fastdiv(gc.n0), make_fastdiv(gc.n1),
                     make_fastdiv(gc.n2));
            IBR_CHECK_LAUNCH();
            continue;
        }
        bool zs = (l > 0) || zero_start;
        if (pre == 0 && zs) IBR_CUDA_TRY(cudaMemsetAsync(U[l], 0, sizeof(T) * C * lev[l].ncell, s));
        for (int it = 0; it < pre; ++it) {
            mg_smooth<T>(lev[l], U[l], Fl(l), C, fld0, sigma, kappa, 0, zs && it == 0, s);
            mg_smooth<T>(lev[l], U[l], Fl(l), C, fld0, sigma, kappa, 1, false, s);
        }
        mg_residual_restrict<T>(lev[l], lev[l + 1], U[l], Fl(l), Fw[l + 1], C, fld0, sigma, kappa, s);
    }
    const bool zs = (lt > 0) || zero_start;
    const int z = zs ? 1 : 0;
    const T sg = (T)sigma;
    if (use_cluster) {
        const long long n0 = lev[lt].ncell;
        ProfScope ps(KID_COARSE, s, 2.0 * C * n0 * sizeof(T));
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[2];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = MG_CL;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.gridDim = dim3(MG_CL * C, 1, 1);
        cfg.blockDim = dim3(1024, 1, 1);
        cfg.dynamicSmemBytes = MG_CL_SMEM;
        cfg.stream = s;
        cfg.attrs = at;
        cfg.numAttrs = pdl_enabled() ? 2 : 1;
        T* ut = U[lt];
        const T* ft = Fl(lt);
        IBR_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_mg_cluster<T>, cl, ut, ft, sg, z, pre, post, coarse_sweeps));
        IBR_CHECK_LAUNCH();
    } else {
        TailLevels tl = make_tail<T>(lev, lt, L, sigma, kappa);
        size_t sm = tail_smem<T>(lev, lt, L);
        long long n0 = lev[lt].ncell;
        int nt = n0 >= 2048 ? 1024 : (int)(((n0 + 1) / 2 + 31) / 32 * 32);
        if (nt < 32) nt = 32;
        ProfScope ps(KID_COARSE, s, 2.0 * C * n0 * sizeof(T));
        mg_set_attributes<T>();
        if (lev[0].d == 3) {
            if (lev[0].wall)
                launch_k(k_mg_tail<3, true, T>, C, nt, sm, s, tl, U[lt], Fl(lt), fld0, sg, z, pre, post,
                                                       coarse_sweeps);
            else
                launch_k(k_mg_tail<3, false, T>, C, nt, sm, s, tl, U[lt], Fl(lt), fld0, sg, z, pre, post,
                                                        coarse_sweeps);
        } else {
            if (lev[0].wall)
                launch_k(k_mg_tail<2, true, T>, C, nt, sm, s, tl, U[lt], Fl(lt), fld0, sg, z, pre, post,
                                                       coarse_sweeps);
            else
                launch_k(k_mg_tail<2, false, T>, C, nt, sm, s, tl, U[lt], Fl(lt), fld0, sg, z, pre, post,
                                                        coarse_sweeps);
        }
        IBR_CHECK_LAUNCH();
    }
    for (int l = lt - 1; l >= 0; --l) {
        if (split(l)) {
            const Geo& g = lev[l];
            T* ru = rbu[l];
            T* rf = rbf[l];
            const T rb_kh2 = (T)(kappa / (g.h * g.h));
            const T rb_inv = rbgs_inv_diag<3, T>((T)sigma, rb_kh2);
            {
                const int nth = (int)((long long)C * g.ncell / (2 * RB_V));
                ProfScope ps(KID_PROLONG, s, (1.0 * g.ncell + lev[l + 1].ncell) * C * sizeof(T));
                launch_k(k_rb_prolong<T>, dim3(grid_1d(nth, 256)), dim3(256), 0, s, ru, (const T*)U[l + 1], g.n0,
                         g.n1, g.n2, nth, make_fastdiv(g.n0 / (2 * RB_V)), make_fastdiv(g.n1), make_fastdiv(g.n2));
                IBR_CHECK_LAUNCH();
            }
            {
                // the post-smoothing half sweeps (the last one also writes u in the
                // natural layout), timed as one sequence
                ProfScope ps(KID_RBGS, s, (3.0 * post + 1.0) * C * g.ncell * sizeof(T), 0.0, 2 * post);
                for (int it = 0; it < post; ++it) {
                    rb_launch_half<T>(g, C, ru, rf, rb_kh2, rb_inv, 1, (T*)nullptr, s);
                    rb_launch_half<T>(g, C, ru, rf, rb_kh2, rb_inv, 0, it + 1 == post ? U[l] : (T*)nullptr, s);
                }
            }
            continue;
        }
        mg_prolong_correct<T>(lev[l], lev[l + 1], U[l], U[l + 1], C, fld0, s);
        for (int it = 0; it < post; ++it) {
            mg_smooth<T>(lev[l], U[l], Fl(l), C, fld0, sigma, kappa, 1, false, s);
            mg_smooth<T>(lev[l], U[l], Fl(l), C, fld0, sigma, kappa, 0, false, s);
        }
    }
}

// Times one V-cycle of each schedule (no cluster; the cluster kernel from
// each feasible level) on the hierarchy lev[0..L) with C stacked fields, on
// the caller's level buffers U[1..L), Fw[1..L) (scratch during the set-up)
// and scratch finest-level arrays, and keeps the fastest for this shape.
// Once per shape and process, outside stream capture; the result of a
// V-cycle does not depend on the schedule (the same arithmetic in the same
// order), only its time.
template <typename T>
void mg_tune_cluster(const Geo* lev, int L, T* const* U, T* const* Fw, int C, int coarse_sweeps, cudaStream_t s) {
    if (lev[0].d != 3 || lev[0].wall || !cluster_ok<T>() || cluster_forced() >= 0) return;
    static const bool off = [] {
        const char* e = std::getenv("IBR_TUNE");
        return e && e[0] == '0';
    }();
    if (off) return;
    const auto key = cl_key(lev, L, C, sizeof(T));
    {
        std::lock_guard<std::mutex> lk(g_cl_mu);
        if (g_cl_top.count(key)) return;
    }
    cudaStreamCaptureStatus cs;
    IBR_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
    if (cs != cudaStreamCaptureStatusNone) return;
    std::vector<int> cands = {-2};
    for (int t = 0; t < L; ++t) {
        ClusterLevels cl;
        int top = 0;
        if (cluster_plan<T>(lev, L, 0.0, 1.0, t, top, cl)) cands.push_back(t);
    }
    if (cands.size() < 2) return;
    const size_t n = (size_t)C * lev[0].ncell;
    T *u0 = nullptr, *f0 = nullptr;
    IBR_CUDA_TRY(cudaMallocAsync(&u0, n * sizeof(T), s));
    IBR_CUDA_TRY(cudaMallocAsync(&f0, n * sizeof(T), s));
    IBR_CUDA_TRY(cudaMemsetAsync(f0, 0, n * sizeof(T), s));
    std::vector<T*> Uv(U, U + L);
    Uv[0] = u0;
    cudaEvent_t e0, e1;
    IBR_CUDA_TRY(cudaEventCreate(&e0));
    IBR_CUDA_TRY(cudaEventCreate(&e1));
    // each candidate: the fastest of three timings of three V-cycles; a
    // cluster schedule must beat the per-level kernels by 5 % to be kept
    int best = -2;
    float best_ms = 1e30f;
    for (int c : cands) {
        {
            std::lock_guard<std::mutex> lk(g_cl_mu);
            g_cl_top[key] = c;
        }
        mg_vcycle<T>(lev, L, Uv.data(), Fw, f0, C, 0, 0.0, 1.0, true, 2, 2, coarse_sweeps, s);
        float ms = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            IBR_CUDA_TRY(cudaEventRecord(e0, s));
            for (int r = 0; r < 3; ++r)
                mg_vcycle<T>(lev, L, Uv.data(), Fw, f0, C, 0, 0.0, 1.0, true, 2, 2, coarse_sweeps, s);
            IBR_CUDA_TRY(cudaEventRecord(e1, s));
            IBR_CUDA_TRY(cudaEventSynchronize(e1));
            float m = 0.f;
            IBR_CUDA_TRY(cudaEventElapsedTime(&m, e0, e1));
            ms = std::min(ms, m);
        }
        if (c != -2) ms *= 1.05f;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    IBR_CUDA_TRY(cudaFreeAsync(u0, s));
    IBR_CUDA_TRY(cudaFreeAsync(f0, s));
    std::lock_guard<std::mutex> lk(g_cl_mu);
    g_cl_top[key] = best;
}

// tuned V-cycle schedule idx: n0, n1, n2, levels, stacked fields, element
// size, first cluster level (-2: none); false past the end
bool tuned_cluster(int idx, int* out7) {
    std::lock_guard<std::mutex> lk(g_cl_mu);
    if (idx < 0 || idx >= (int)g_cl_top.size()) return false;
    auto it = g_cl_top.begin();
    std::advance(it, idx);
    for (int q = 0; q < 6; ++q) out7[q] = (int)it->first[q];
    out7[6] = it->second;
    return true;
}

template <typename T>
void ps_divergence(const Geo& g, const T* y, const T* hd, T* q_rhs, double rhs_scale, T* q, cudaStream_t s) {
    dim3 grid((g.n0 + BX - 1) / BX, (g.n1 + BY - 1) / BY, g.n2), blk(BX, BY);
    ProfScope ps(KID_PS_DIV, s, (g.d + 3.0) * g.ncell * sizeof(T));
    const T ih = (T)(1.0 / g.h), rs = (T)rhs_scale;
    if (g.d == 3) {
        if (g.wall)
            launch_k(k_ps_div<3, true, T>, grid, blk, 0, s, y, hd, q_rhs, rs, q, g, ih);
        else
            launch_k(k_ps_div<3, false, T>, grid, blk, 0, s, y, hd, q_rhs, rs, q, g, ih);
    } else {
        if (g.wall)
            launch_k(k_ps_div<2, true, T>, grid, blk, 0, s, y, hd, q_rhs, rs, q, g, ih);
        else
            launch_k(k_ps_div<2, false, T>, grid, blk, 0, s, y, hd, q_rhs, rs, q, g, ih);
    }
    IBR_CHECK_LAUNCH();
}

template <typename T>
void ps_finish(const Geo& g, const T* y, const T* phi, const T* q, T* z, double c_q, double c_phi,
               cudaStream_t s) {
    dim3 grid((g.n0 + BX - 1) / BX, (g.n1 + BY - 1) / BY, g.n2), blk(BX, BY);
    ProfScope ps(KID_PS_FINISH, s, (2.0 * g.d + 3.0) * g.ncell * sizeof(T));
    const T h = (T)g.h, cq = (T)c_q, cp = (T)c_phi;
    if (g.d == 3) {
        if (g.wall)
            launch_k(k_ps_finish<3, true, T>, grid, blk, 0, s, y, phi, q, z, g, h, cq, cp);
        else
            launch_k(k_ps_finish<3, false, T>, grid, blk, 0, s, y, phi, q, z, g, h, cq, cp);
    } else {
        if (g.wall)
            launch_k(k_ps_finish<2, true, T>, grid, blk, 0, s, y, phi, q, z, g, h, cq, cp);
        else
            launch_k(k_ps_finish<2, false, T>, grid, blk, 0, s, y, phi, q, z, g, h, cq, cp);
    }
    IBR_CHECK_LAUNCH();
}

void wall_lift(const Geo& g, int a, int side, const double* data, double* b, double eta, cudaStream_t s) {
    const int ns[3] = {g.n0, g.n1, g.n2};
    long long nf = g.ncell / ns[a];
    ProfScope ps(KID_SMALL, s, 0.0);
    k_wall_lift<<<grid_1d(nf, 128), 128, 0, s>>>(g, a, side, data, b, eta / (g.h * g.h), 1.0 / g.h);
    IBR_CHECK_LAUNCH();
}

#define IBR_INST(T)                                                                                        \
    template void stokes_apply<T>(const Geo&, const T*, T*, double, double, const double*, cudaStream_t); \
    template void mg_smooth<T>(const Geo&, T*, const T*, int, int, double, double, int, bool, cudaStream_t); \
    template void mg_residual_restrict<T>(const Geo&, const Geo&, const T*, const T*, T*, int, int, double, \
                                          double, cudaStream_t);                                          \
    template void mg_prolong_correct<T>(const Geo&, const Geo&, T*, const T*, int, int, cudaStream_t);    \
    template void mg_coarse_solve<T>(const Geo&, T*, const T*, int, int, double, double, int, cudaStream_t); \
    template void mg_set_attributes<T>();                                                                   \
    template void mg_tune_smoother<T>(const Geo&, int, cudaStream_t);                                       \
    template void mg_tune_cluster<T>(const Geo*, int, T* const*, T* const*, int, int, cudaStream_t);          \
    template void mg_vcycle<T>(const Geo*, int, T* const*, T* const*, const T*, int, int, double, double, bool, \
                               int, int, int, cudaStream_t, T*, T*, T*, T*);                                \
    template void ps_divergence<T>(const Geo&, const T*, const T*, T*, double, T*, cudaStream_t);         \
    template void ps_finish<T>(const Geo&, const T*, const T*, const T*, T*, double, double, cudaStream_t);
IBR_INST(double)
IBR_INST(float)
#undef IBR_INST

}  // namespace ibr
