// Approximate mobility M~ (Sec. IV, Eq. M_tilde_ij) and its dense solve
// (Sec. V.C): build per body, Cholesky factor, explicit inverse, so that
// each preconditioner application is one block-diagonal matrix-vector product.
//
// The factorisation is a blocked right-looking Cholesky on 32x32 tiles
// (diagonal tile factor + inverse in shared memory, panel = A_ik X_kk^T,
// trailing rank-32 update), then X = L^-1 tile by tile, then M^-1 = X^T X.
#include <type_traits>

#include "ibr_internal.cuh"

namespace ibr {
namespace {

constexpr int TB = 32;

__device__ __forceinline__ void mob_fg(const MobParams& p, double r, double& f, double& g) {
    if (p.model == IBR_MOB_RPY) {
        // Eq. RPYTensor, minus the periodic correction of App. A on f
        double a = p.a;
        double c = 1.0 / (6.0 * M_PI * p.eta * a);
        if (r > 2.0 * a) {
            double ar = a / r, ar3 = ar * ar * ar;
            f = c * (0.75 * ar + 0.5 * ar3);
            g = c * (0.75 * ar - 1.5 * ar3);
        } else {
            f = c * (1.0 - 9.0 * r / (32.0 * a));
            g = c * (3.0 * r / (32.0 * a));
        }
        f -= p.corr;
    } else {
        // App. B steady 2-D: f = f(0) - f~(r/h)/(4 pi eta), g = g~(r/h)/(4 pi eta)
        const double* k = p.coef;
        double x = r / p.h;
        double lx = x > 0.0 ? log(x) : 0.0;
        double x2 = x * x, x3 = x2 * x;
        double ft = (k[0] * x2 + k[1] * x3 + k[2] * x3 * lx) / (1.0 + k[3] * x + k[4] * x2 + k[2] * x3);
        double gt = (k[5] * x2 + k[6] * x3) / (1.0 + k[7] * x + k[8] * x2 + k[6] * x3);
        double f0 = log(p.l / (3.708 * p.a)) / (4.0 * M_PI * p.eta);
        f = f0 - ft / (4.0 * M_PI * p.eta);
        g = gt / (4.0 * M_PI * p.eta);
    }
}

template <int D>
__global__ void k_mtilde(int Nb, const double* __restrict__ rel, MobParams p, double* __restrict__ M) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)Nb * Nb) return;
    int i = (int)(t / Nb), j = (int)(t % Nb);
    double rv[3] = {0, 0, 0};
    double r2 = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        rv[a] = rel[i * D + a] - rel[j * D + a];
        if (p.box[a] > 0.0) rv[a] -= p.box[a] * rint(rv[a] / p.box[a]);
        r2 += rv[a] * rv[a];
    }
    double r = sqrt(r2);
    double f, g;
    mob_fg(p, r, f, g);
    long long ld = (long long)Nb * D;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) {
            double v = (a == b ? f : 0.0);
            if (r > 0.0) v += g * rv[a] * rv[b] / r2;
            M[(long long)(i * D + a) * ld + j * D + b] = v;
        }
}

// element (r, c) of the zero/identity-padded tile view of an n x n matrix
template <typename T>
__device__ __forceinline__ T ld_pad(const T* A, int n, int r, int c) {
    if (r < n && c < n) return A[(long long)r * n + c];
    return r == c ? T(1) : T(0);
}

// factor the diagonal tile k in place (lower), write its inverse to Dinv[k]
template <typename T>
__global__ void __launch_bounds__(TB * TB) k_potrf_diag(int n, T* A, int k, T* Dinv, int* info, T min_pivot) {
    __shared__ T a[TB][TB + 1];
    __shared__ T x[TB][TB + 1];
    int tr = threadIdx.y, tc = threadIdx.x;
    int r0 = k * TB;
    a[tr][tc] = ld_pad(A, n, r0 + tr, r0 + tc);
    x[tr][tc] = T(0);
    __syncthreads();
    for (int c = 0; c < TB; ++c) {
        if (tr == c && tc == c) {
            T d = a[c][c];
            if (!(d > min_pivot)) {
                if (info) atomicCAS(info, 0, r0 + c + 1);
                d = T(1);
            }
            a[c][c] = sqrt(d);
        }
        __syncthreads();
        if (tc == c && tr > c) a[tr][c] /= a[c][c];
        __syncthreads();
        if (tr > c && tc > c && tc <= tr) a[tr][tc] -= a[tr][c] * a[tc][c];
        __syncthreads();
    }
    // X = L^-1: thread column tc (tr == 0) does forward substitution
    if (tr == 0) {
        int j = tc;
        x[j][j] = T(1) / a[j][j];
        for (int i = j + 1; i < TB; ++i) {
            T s = T(0);
            for (int l = j; l < i; ++l) s += a[i][l] * x[l][j];
            x[i][j] = -s / a[i][i];
        }
    }
    __syncthreads();
    if (r0 + tr < n && r0 + tc < n) A[(long long)(r0 + tr) * n + r0 + tc] = tc <= tr ? a[tr][tc] : T(0);
    Dinv[(long long)k * TB * TB + tr * TB + tc] = x[tr][tc];
}

// L_ik = A_ik X_kk^T for every tile row i > k (blockIdx.x = i - k - 1)
template <typename T>
__global__ void __launch_bounds__(TB * TB) k_trsm_panel(int n, T* A, int k, const T* Dinv) {
    __shared__ T a[TB][TB + 1];
    __shared__ T x[TB][TB + 1];
    int i = k + 1 + blockIdx.x;
    int tr = threadIdx.y, tc = threadIdx.x;
    a[tr][tc] = ld_pad(A, n, i * TB + tr, k * TB + tc);
    x[tr][tc] = Dinv[(long long)k * TB * TB + tr * TB + tc];
    __syncthreads();
    T s = T(0);
    for (int l = 0; l < TB; ++l) s += a[tr][l] * x[tc][l];
    int r = i * TB + tr, c = k * TB + tc;
    if (r < n && c < n) A[(long long)r * n + c] = s;
}

// A_ij -= L_ik L_jk^T for k < j <= i (lower tiles), blockIdx.x enumerates (i, j)
template <typename T>
__global__ void __launch_bounds__(TB * TB) k_syrk(int n, T* A, int k, int nb) {
    __shared__ T li[TB][TB + 1];
    __shared__ T lj[TB][TB + 1];
    int t = blockIdx.x;
    // t -> (ii, jj) with 0 <= jj <= ii < m, row-major over the lower triangle
    int ii = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while ((ii + 1) * (ii + 2) / 2 <= t) ++ii;
    while (ii * (ii + 1) / 2 > t) --ii;
    int jj = t - ii * (ii + 1) / 2;
    int i = k + 1 + ii, j = k + 1 + jj;
    int tr = threadIdx.y, tc = threadIdx.x;
    int kc = k * TB + tc;
    li[tr][tc] = (i * TB + tr < n && kc < n) ? A[(long long)(i * TB + tr) * n + kc] : T(0);
    lj[tr][tc] = (j * TB + tr < n && kc < n) ? A[(long long)(j * TB + tr) * n + kc] : T(0);
    __syncthreads();
    T s = T(0);
    for (int l = 0; l < TB; ++l) s += li[tr][l] * lj[tc][l];
    int r = i * TB + tr, c = j * TB + tc;
    if (r < n && c < n) A[(long long)r * n + c] -= s;
}

// X_ik = -X_ii sum_{j=k}^{i-1} L_ij X_jk for all k < i (blockIdx.x = k); X in W
template <typename T>
__global__ void __launch_bounds__(TB * TB) k_trinv_row(int n, const T* A, T* W, int i, const T* Dinv) {
    __shared__ T l[TB][TB + 1];
    __shared__ T xx[TB][TB + 1];
    int k = blockIdx.x;
    int tr = threadIdx.y, tc = threadIdx.x;
    T s = T(0);
    for (int j = k; j < i; ++j) {
        l[tr][tc] = ld_pad(A, n, i * TB + tr, j * TB + tc);
        // X_jk (diagonal tile of X when j == k comes from Dinv)
        if (j == k)
            xx[tr][tc] = Dinv[(long long)k * TB * TB + tr * TB + tc];
        else
            xx[tr][tc] = (j * TB + tr < n && k * TB + tc < n) ? W[(long long)(j * TB + tr) * n + k * TB + tc] : T(0);
        __syncthreads();
        for (int q = 0; q < TB; ++q) s += l[tr][q] * xx[q][tc];
        __syncthreads();
    }
    // multiply by -X_ii
    l[tr][tc] = Dinv[(long long)i * TB * TB + tr * TB + tc];
    xx[tr][tc] = s;
    __syncthreads();
    T o = T(0);
    for (int q = 0; q < TB; ++q) o -= l[tr][q] * xx[q][tc];
    int r = i * TB + tr, c = k * TB + tc;
    if (r < n && c < n) W[(long long)r * n + c] = o;
}

// copy the diagonal X tiles into W (so that W holds the full lower X)
template <typename T>
__global__ void __launch_bounds__(TB * TB) k_put_diag(int n, T* W, const T* Dinv) {
    int k = blockIdx.x;
    int tr = threadIdx.y, tc = threadIdx.x;
    int r = k * TB + tr, c = k * TB + tc;
    if (r < n && c < n) W[(long long)r * n + c] = tc <= tr ? Dinv[(long long)k * TB * TB + tr * TB + tc] : T(0);
}

// M^-1 tile (a, b) = sum_{c >= max(a,b)} X_ca^T X_cb   (X lower, in W)
template <typename T>
__global__ void __launch_bounds__(TB * TB) k_xtx(int n, const T* W, T* M, int nb) {
    __shared__ T xa[TB][TB + 1];
    __shared__ T xb[TB][TB + 1];
    int a = blockIdx.x, b = blockIdx.y;
    int tr = threadIdx.y, tc = threadIdx.x;
    T s = T(0);
    int c0 = a > b ? a : b;
    for (int c = c0; c < nb; ++c) {
        int row = c * TB + tr;
        xa[tr][tc] = (row < n && a * TB + tc < n && a * TB + tc <= row) ? W[(long long)row * n + a * TB + tc] : T(0);
        xb[tr][tc] = (row < n && b * TB + tc < n && b * TB + tc <= row) ? W[(long long)row * n + b * TB + tc] : T(0);
        __syncthreads();
        for (int q = 0; q < TB; ++q) s += xa[q][tr] * xb[q][tc];
        __syncthreads();
    }
    int r = a * TB + tr, c = b * TB + tc;
    if (r < n && c < n) M[(long long)r * n + c] = s;
}

// periodic window of component al at point p (lab coordinates in [0, L)):
// per axis b the first of the KW nodes and their weights (face al sits at
// integer positions along al and half-integer positions along the others)
template <int D, int KW>
__device__ __forceinline__ void pair_window(const Geo& g, const double* p, int al, int* j0, double (*w)[KW]) {
#pragma unroll
    for (int b = 0; b < D; ++b) {
        const double sb = p[b] / g.h - (al == b ? 0.0 : 0.5);
        kernel_window(KW, sb, j0[b], w[b]);
    }
}

// one thread per unordered pair (i <= j; 16 x 16 blocks, those wholly below
// the diagonal exit): it forms M~_ij and writes it and its transpose M~_ji
// the same window with FP32 weights (the table is FP32): the position and
// its offset from the window's first node stay FP64, the kernel value and the
// KW^d-cell sums of the M~ build run on the FP32 pipe (the six-point weights
// are formed in FP64 and rounded)
__device__ __forceinline__ float peskin4f(float r) {
    r = fabsf(r);
    if (r < 1.0f) return 0.125f * (3.0f - 2.0f * r + sqrtf(1.0f + 4.0f * r - 4.0f * r * r));
    if (r < 2.0f) return 0.125f * (5.0f - 2.0f * r - sqrtf(fmaxf(-7.0f + 12.0f * r - 4.0f * r * r, 0.0f)));
    return 0.0f;
}

template <int D, int KW>
__device__ __forceinline__ void pair_window_f(const Geo& g, const double* p, int al, int* j0, float (*w)[KW]) {
#pragma unroll
    for (int b = 0; b < D; ++b) {
        const double sb = p[b] / g.h - (al == b ? 0.0 : 0.5);
        const double fl = floor(sb);
        if (KW == 6) {
            double w6[6];
            j0[b] = (int)fl - 2;
            bkp6_weights(sb - fl, w6);
#pragma unroll
            for (int m = 0; m < KW; ++m) w[b][m] = (float)w6[m];
        } else {
            j0[b] = (int)fl - 1;
            const float fr = (float)(sb - fl);  // in [0, 1)
#pragma unroll
            for (int m = 0; m < KW; ++m) w[b][m] = peskin4f(fr + 1.0f - (float)m);
        }
    }
}

template <int D, int KW>
__global__ void __launch_bounds__(256) k_pair_mtilde(Geo g, int nr, const double* __restrict__ q, int S,
                                                     const double* __restrict__ x0, const float* __restrict__ tab,
                                                     double* __restrict__ M) {
    if (blockIdx.x < blockIdx.y) return;
    const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
    if (i >= nr || j >= nr || j < i) return;
    const int ns[3] = {g.n0, g.n1, g.n2};
    // acc[0]: sum_s T_s(q_i - q_j);  acc[1]: sum_s T_s(q_j - q_i)^T
    double acc[2][D][D];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) acc[0][a][b] = acc[1][a][b] = 0.0;
    for (int tr = 0; tr < 2; ++tr) {
        // tr = 0: T(q_i - q_j)^{ab};  tr = 1: T(q_j - q_i)^{ba}
        const int u = tr ? j : i, v = tr ? i : j;
        for (int s = 0; s < S; ++s) {
            double p[D];
#pragma unroll
            for (int b = 0; b < D; ++b) {
                const double Lb = ns[b] * g.h;
                double x = x0[s * D + b] + q[(long long)u * D + b] - q[(long long)v * D + b];
                x -= Lb * floor(x / Lb);
                if (x >= Lb) x -= Lb;
                p[b] = x;
            }
#pragma unroll
            for (int al = 0; al < D; ++al) {
                int j0[D];
                float w[D][KW];
                pair_window_f<D, KW>(g, p, al, j0, w);
                float sum[D];
#pragma unroll
                for (int be = 0; be < D; ++be) sum[be] = 0.0f;
                const int S_win = D == 3 ? KW * KW * KW : KW * KW;
                for (int c = 0; c < S_win; ++c) {
                    long long cell = 0, stride = 1;
                    float wt = 1.0f;
                    int cc = c;
#pragma unroll
                    for (int b = 0; b < D; ++b) {
                        const int m = cc % KW;
                        cc /= KW;
                        int jj = (j0[b] + m) % ns[b];
                        if (jj < 0) jj += ns[b];
                        cell += jj * stride;
                        stride *= ns[b];
                        wt *= w[b][m];
                    }
#pragma unroll
                    for (int be = 0; be < D; ++be)
                        sum[be] = fmaf(wt, tab[((long long)(s * D + be) * D + al) * g.ncell + cell], sum[be]);
                }
#pragma unroll
                for (int be = 0; be < D; ++be) {
                    if (tr == 0)
                        acc[0][al][be] += (double)sum[be];
                    else
                        acc[1][be][al] += (double)sum[be];
                }
            }
        }
    }
    const double sc = 0.5 / S;
    const long long ld = (long long)nr * D;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int b = 0; b < D; ++b) {
            const double v = sc * (acc[0][a][b] + acc[1][a][b]);
            M[((long long)i * D + a) * ld + (long long)j * D + b] = v;
            M[((long long)j * D + b) * ld + (long long)i * D + a] = v;  // exactly symmetric
        }
}

template <int D, int KW>
__global__ void k_point_spread(Geo g, const double* __restrict__ x0, int beta, double scale, double* __restrict__ y) {
    const int c = threadIdx.x;
    if (c >= (D == 3 ? KW * KW * KW : KW * KW)) return;
    const int ns[3] = {g.n0, g.n1, g.n2};
    int j0[D];
    double w[D][KW];
    pair_window<D, KW>(g, x0, beta, j0, w);
    long long cell = 0, stride = 1;
    double wt = 1.0;
    int cc = c;
#pragma unroll
    for (int b = 0; b < D; ++b) {
        const int m = cc % KW;
        cc /= KW;
        int jj = (j0[b] + m) % ns[b];
        if (jj < 0) jj += ns[b];
        cell += jj * stride;
        stride *= ns[b];
        wt *= w[b][m];
    }
    y[(long long)beta * g.ncell + cell] = scale * wt;
}

template <typename T>
__global__ void k_add_diag(int n, T* M, T delta) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) M[(long long)i * n + i] += delta;
}

template <typename Ti, typename To>
__global__ void k_mat_convert(long long n, const Ti* __restrict__ a, To* __restrict__ b) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = (To)a[i];
}

// one warp per output row; body block b spans rows [roff[b], roff[b+1])
template <typename T, typename Tv>
__global__ void k_bd_gemv(int B, const long long* __restrict__ moff, const int* __restrict__ roff, const T* __restrict__ M,
                          const Tv* __restrict__ rhs, Tv* __restrict__ out) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    int total = roff[B];
    if (warp >= total) return;
    int b = 0;
    while (roff[b + 1] <= warp) ++b;
    int r0 = roff[b], nr = roff[b + 1] - r0;
    int row = warp - r0;
    const T* Mr = M + moff[b] + (long long)row * nr;
    double acc = 0.0;
    if constexpr (std::is_same<T, float>::value && std::is_same<Tv, float>::value) {
        // FP32 path: per-lane FP32 sums (FP64 arithmetic runs at a small
        // fraction of the FP32 rate on this part), combined in FP64 across
        // lanes; four independent partial sums per lane
        const float* Mf = reinterpret_cast<const float*>(Mr);
        const float* xf = reinterpret_cast<const float*>(rhs) + r0;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        int c = lane;
        for (; c + 96 < nr; c += 128) {
            a0 = fmaf(Mf[c], xf[c], a0);
            a1 = fmaf(Mf[c + 32], xf[c + 32], a1);
            a2 = fmaf(Mf[c + 64], xf[c + 64], a2);
            a3 = fmaf(Mf[c + 96], xf[c + 96], a3);
        }
        for (; c < nr; c += 32) a0 = fmaf(Mf[c], xf[c], a0);
        acc = ((double)a0 + (double)a1) + ((double)a2 + (double)a3);
    } else {
        for (int c = lane; c < nr; c += 32) acc += (double)Mr[c] * (double)rhs[r0 + c];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[warp] = (Tv)acc;
}

}  // namespace

void mtilde_build(int d, int Nb, const double* rel_b, const MobParams& p, double* M, cudaStream_t s) {
    long long n = (long long)Nb * Nb;
    ProfScope ps(KID_MTILDE, s, (double)n * d * d * 8);
    if (d == 3)
        k_mtilde<3><<<grid_1d(n, 256), 256, 0, s>>>(Nb, rel_b, p, M);
    else
        k_mtilde<2><<<grid_1d(n, 256), 256, 0, s>>>(Nb, rel_b, p, M);
    IBR_CHECK_LAUNCH();
}

void pair_mtilde(const Geo& g, int nr, const double* q, int S, const double* x0, const float* tab, double* M,
                 cudaStream_t s) {
    const long long n = (long long)nr * nr;
    ProfScope ps(KID_MTILDE, s, (double)n * g.d * g.d * 8);
    const int nt = (nr + 15) / 16;
    dim3 grid(nt, nt), blk(16, 16);
    if (g.d == 3) {
        if (g.kw == 6)
            k_pair_mtilde<3, 6><<<grid, blk, 0, s>>>(g, nr, q, S, x0, tab, M);
        else
            k_pair_mtilde<3, 4><<<grid, blk, 0, s>>>(g, nr, q, S, x0, tab, M);
    } else {
        if (g.kw == 6)
            k_pair_mtilde<2, 6><<<grid, blk, 0, s>>>(g, nr, q, S, x0, tab, M);
        else
            k_pair_mtilde<2, 4><<<grid, blk, 0, s>>>(g, nr, q, S, x0, tab, M);
    }
    IBR_CHECK_LAUNCH();
}

void point_spread(const Geo& g, const double* x0, int beta, double scale, double* y, cudaStream_t s) {
    if (g.d == 3) {
        if (g.kw == 6)
            k_point_spread<3, 6><<<1, 256, 0, s>>>(g, x0, beta, scale, y);
        else
            k_point_spread<3, 4><<<1, 64, 0, s>>>(g, x0, beta, scale, y);
    } else {
        if (g.kw == 6)
            k_point_spread<2, 6><<<1, 64, 0, s>>>(g, x0, beta, scale, y);
        else
            k_point_spread<2, 4><<<1, 16, 0, s>>>(g, x0, beta, scale, y);
    }
    IBR_CHECK_LAUNCH();
}

template <typename T>
void spd_inverse(int n, T* M, T* work, int* info_dev, double min_pivot, cudaStream_t s) {
    int nb = (n + TB - 1) / TB;
    ProfScope ps(KID_SPD_INV, s, 2.0 * n * n * sizeof(T));
    T* Dinv = nullptr;
    IBR_CUDA_TRY(cudaMallocAsync(&Dinv, (size_t)nb * TB * TB * sizeof(T), s));
    dim3 tile(TB, TB);
    for (int k = 0; k < nb; ++k) {
        k_potrf_diag<T><<<1, tile, 0, s>>>(n, M, k, Dinv, info_dev, (T)min_pivot);
        IBR_CHECK_LAUNCH();
        int m = nb - k - 1;
        if (m > 0) {
            k_trsm_panel<T><<<m, tile, 0, s>>>(n, M, k, Dinv);
            IBR_CHECK_LAUNCH();
            k_syrk<T><<<m * (m + 1) / 2, tile, 0, s>>>(n, M, k, nb);
            IBR_CHECK_LAUNCH();
        }
    }
    // X = L^-1 into work (lower); diagonal tiles from Dinv
    IBR_CUDA_TRY(cudaMemsetAsync(work, 0, (size_t)n * n * sizeof(T), s));
    k_put_diag<T><<<nb, tile, 0, s>>>(n, work, Dinv);
    IBR_CHECK_LAUNCH();
    for (int i = 1; i < nb; ++i) {
        k_trinv_row<T><<<i, tile, 0, s>>>(n, M, work, i, Dinv);
        IBR_CHECK_LAUNCH();
    }
    k_xtx<T><<<dim3(nb, nb), tile, 0, s>>>(n, work, M, nb);
    IBR_CHECK_LAUNCH();
    IBR_CUDA_TRY(cudaFreeAsync(Dinv, s));
}

template <typename T>
void add_diag(int n, T* M, double delta, cudaStream_t s) {
    ProfScope ps(KID_SPD_INV, s, 0.0);
    k_add_diag<T><<<grid_1d(n, 256), 256, 0, s>>>(n, M, (T)delta);
    IBR_CHECK_LAUNCH();
}

template <typename Ti, typename To>
void mat_convert(long long n, const Ti* a, To* b, cudaStream_t s) {
    ProfScope ps(KID_SPD_INV, s, (double)n * (sizeof(Ti) + sizeof(To)));
    k_mat_convert<Ti, To><<<grid_1d(n, 256) > 4096 ? 4096 : grid_1d(n, 256), 256, 0, s>>>(n, a, b);
    IBR_CHECK_LAUNCH();
}

template <typename T, typename Tv>
void blockdiag_gemv(int B, const long long* moff_dev, const int* roff_dev, int total_rows, const T* Mall, const Tv* rhs,
                    Tv* out, cudaStream_t s) {
    int threads = 256;
    int blocks = grid_1d((long long)total_rows * 32, threads);
    ProfScope ps(KID_GEMV, s, (double)total_rows * total_rows * sizeof(T));
    k_bd_gemv<T, Tv><<<blocks, threads, 0, s>>>(B, moff_dev, roff_dev, Mall, rhs, out);
    IBR_CHECK_LAUNCH();
}

template void spd_inverse<double>(int, double*, double*, int*, double, cudaStream_t);
template void spd_inverse<float>(int, float*, float*, int*, double, cudaStream_t);
template void add_diag<double>(int, double*, double, cudaStream_t);
template void add_diag<float>(int, float*, double, cudaStream_t);
template void mat_convert<double, float>(long long, const double*, float*, cudaStream_t);
template void mat_convert<double, double>(long long, const double*, double*, cudaStream_t);
template void blockdiag_gemv<double, double>(int, const long long*, const int*, int, const double*, const double*,
                                             double*, cudaStream_t);
template void blockdiag_gemv<float, float>(int, const long long*, const int*, int, const float*, const float*, float*,
                                           cudaStream_t);

}  // namespace ibr
