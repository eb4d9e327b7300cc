// Vector kernels of the Krylov solvers (Sec. V: FGMRES outer, GMRES(N_s) inner).
// Dot products use a fixed grid and a fixed-order final sum, so results are
// bitwise reproducible run to run.
#include <type_traits>

#include "ibr_internal.cuh"

namespace ibr {
namespace {

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block-reduce NV values per thread into out[0..NV) by thread 0 (double)
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* out) {
    __shared__ double sm[RED_THREADS / 32][NV];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double s = warp_sum(v[q]);
        if (lane == 0) sm[wid][q] = s;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double s = lane < RED_THREADS / 32 ? sm[lane][q] : 0.0;
            s = warp_sum(s);
            if (lane == 0) out[q] = s;
        }
    }
    __syncthreads();
}

// block-reduce the first nq of NV values per thread into out[0..nq) (thread 0
// writes): the warp stage in the accumulator type TA (FP32 sums stay on the
// FP32 pipe; FP64 runs at 1/64 of its rate on this part), the cross-warp
// stage in double; fixed order, so bitwise reproducible
template <typename TA, int NV>
__device__ __forceinline__ void block_sum_t(TA (&v)[NV], int nq, double* out) {
    __shared__ double sm[RED_THREADS / 32][NV];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        if (q < nq) {
            TA x = v[q];
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) sm[wid][q] = (double)x;
        }
    }
    __syncthreads();
    if (threadIdx.x < nq) {
        double acc = 0.0;
#pragma unroll
        for (int w = 0; w < RED_THREADS / 32; ++w) acc += sm[w][threadIdx.x];
        out[threadIdx.x] = acc;
    }
    __syncthreads();
}

template <typename T>
__global__ void k_axpby(long long n, T a, const T* __restrict__ x, T b, T* __restrict__ y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = a * x[i] + b * y[i];
}

template <typename T>
__global__ void k_scale_copy(long long n, const double* __restrict__ sc, int invert, const T* __restrict__ x,
                             T* __restrict__ y) {
    __shared__ T as;
    if (threadIdx.x == 0) {
        const double s = *sc;
        as = (T)(invert ? (s != 0.0 ? 1.0 / s : 0.0) : s);
    }
    __syncthreads();
    const T a = as;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = a * x[i];
}

template <typename Ti, typename To>
__global__ void k_convert(long long n, const Ti* __restrict__ x, To* __restrict__ y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = (To)x[i];
}

// partial[blk*k + j] = sum over this block's elements of V_j . w, j in [j0, j0+CH)
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_mdot(long long n, const T* __restrict__ V, long long ld, int k,
                                                      const T* __restrict__ w, double* __restrict__ partial) {
    for (int j0 = 0; j0 < k; j0 += MDOT_CHUNK) {
        T tacc[MDOT_CHUNK];
#pragma unroll
        for (int q = 0; q < MDOT_CHUNK; ++q) tacc[q] = T(0);
        int nq = min(MDOT_CHUNK, k - j0);
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
             i += (long long)gridDim.x * blockDim.x) {
            T wi = w[i];
#pragma unroll
            for (int q = 0; q < MDOT_CHUNK; ++q)
                if (q < nq) tacc[q] += V[(long long)(j0 + q) * ld + i] * wi;
        }
        __shared__ double outv[MDOT_CHUNK];
        block_sum_t<T, MDOT_CHUNK>(tacc, nq, outv);
        if (threadIdx.x < nq) partial[(long long)blockIdx.x * k + j0 + threadIdx.x] = outv[threadIdx.x];
        __syncthreads();
    }
}

// out[j] = sum_blk partial[blk*k + j]   (grid: k blocks)
__global__ void k_finalize(const double* __restrict__ partial, int nblk, int k, double* __restrict__ out) {
    int j = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partial[(long long)b * k + j];
    double v[1] = {s};
    __shared__ double o[1];
    block_sum<1>(v, o);
    if (threadIdx.x == 0) out[j] = o[0];
}

// w -= sum_j h_j V_j ; then partial dots V_j . w (second CGS pass)
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_update_mdot(long long n, const T* __restrict__ V, long long ld,
                                                             int k, const double* __restrict__ h,
                                                             T* __restrict__ w, double* __restrict__ partial) {
    __shared__ T hs[128];
    for (int j = threadIdx.x; j < k; j += blockDim.x) hs[j] = (T)h[j];
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        T s = T(0);
        for (int j = 0; j < k; ++j) s += hs[j] * V[(long long)j * ld + i];
        w[i] = w[i] - s;
    }
    // the elements this thread wrote are re-read by the same thread below
    for (int j0 = 0; j0 < k; j0 += MDOT_CHUNK) {
        T tacc[MDOT_CHUNK];
#pragma unroll
        for (int q = 0; q < MDOT_CHUNK; ++q) tacc[q] = T(0);
        int nq = min(MDOT_CHUNK, k - j0);
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
             i += (long long)gridDim.x * blockDim.x) {
            T wi = w[i];
#pragma unroll
            for (int q = 0; q < MDOT_CHUNK; ++q)
                if (q < nq) tacc[q] += V[(long long)(j0 + q) * ld + i] * wi;
        }
        __shared__ double outv[MDOT_CHUNK];
        block_sum_t<T, MDOT_CHUNK>(tacc, nq, outv);
        if (threadIdx.x < nq) partial[(long long)blockIdx.x * k + j0 + threadIdx.x] = outv[threadIdx.x];
        __syncthreads();
    }
}

// w -= sum_j h_j V_j ; partial |w|^2
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_update_norm(long long n, const T* __restrict__ V, long long ld,
                                                             int k, const double* __restrict__ h,
                                                             T* __restrict__ w, double* __restrict__ partial) {
    __shared__ T hs[128];
    for (int j = threadIdx.x; j < k; j += blockDim.x) hs[j] = (T)h[j];
    __syncthreads();
    T acc = T(0);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        T s = T(0);
        for (int j = 0; j < k; ++j) s += hs[j] * V[(long long)j * ld + i];
        T wi = w[i] - s;
        w[i] = wi;
        acc += wi * wi;
    }
    T v[1] = {acc};
    __shared__ double o[1];
    block_sum_t<T, 1>(v, 1, o);
    if (threadIdx.x == 0) partial[blockIdx.x] = o[0];
}

template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_norm2(long long n, const T* __restrict__ w,
                                                       double* __restrict__ partial) {
    T acc = T(0);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        T wi = w[i];
        acc += wi * wi;
    }
    T v[1] = {acc};
    __shared__ double o[1];
    block_sum_t<T, 1>(v, 1, o);
    if (threadIdx.x == 0) partial[blockIdx.x] = o[0];
}

// x (+)= sum_j y_j Z_j, accumulated in the wider of T and Tz (an FP32
// combination stays on the FP32 pipe)
template <typename T, typename Tz>
__global__ void k_combine(long long n, const Tz* __restrict__ Z, long long ld, int k, const double* __restrict__ y,
                          T* __restrict__ x, int accumulate) {
    using TA = typename std::conditional<(sizeof(T) > sizeof(Tz)), T, Tz>::type;
    __shared__ TA ys[128];
    for (int j = threadIdx.x; j < k; j += blockDim.x) ys[j] = (TA)y[j];
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        TA s = accumulate ? (TA)x[i] : TA(0);
        for (int j = 0; j < k; ++j) s += ys[j] * (TA)Z[(long long)j * ld + i];
        x[i] = (T)s;
    }
}

// partial[blk*C + c] = sum of block c's elements handled by this CTA
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_block_sums(long long m, int C, const T* __restrict__ x,
                                                            double* __restrict__ partial) {
    for (int c = 0; c < C; ++c) {
        T tacc = T(0);
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m;
             i += (long long)gridDim.x * blockDim.x)
            tacc += x[(long long)c * m + i];
        T v[1] = {tacc};
        __shared__ double o[1];
        block_sum_t<T, 1>(v, 1, o);
        if (threadIdx.x == 0) partial[(long long)blockIdx.x * C + c] = o[0];
    }
}

__global__ void k_scale_vals(int C, double s, double* v) {
    int c = threadIdx.x;
    if (c < C) v[c] *= s;
}

// component c = blockIdx.y
template <typename T>
__global__ void k_subtract_means(long long m, T* __restrict__ x, const double* __restrict__ means) {
    const T mu = (T)means[blockIdx.y];
    x += (long long)blockIdx.y * m;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x)
        x[i] -= mu;
}

// ---- small FP64 bookkeeping kernels (one thread) --------------------------
__global__ void k_arnoldi_column(double* H, int ldh, const double* h1, const double* h2, const double* nrm2, int j,
                                 double* cs, double* sn, double* gv, double* res_out, double* inv_norm_out) {
    double* col = H + (long long)j * ldh;
    for (int i = 0; i <= j; ++i) col[i] = h1[i] + (h2 ? h2[i] : 0.0);
    double nr = sqrt(fmax(*nrm2, 0.0));
    col[j + 1] = nr;
    *inv_norm_out = nr > 0.0 ? 1.0 / nr : 0.0;
    for (int i = 0; i < j; ++i) {
        double a = col[i], b = col[i + 1];
        col[i] = cs[i] * a + sn[i] * b;
        col[i + 1] = -sn[i] * a + cs[i] * b;
    }
    double a = col[j], b = col[j + 1];
    double r = hypot(a, b);
    double c = 1.0, s = 0.0;
    if (r > 0.0) {
        c = a / r;
        s = b / r;
    }
    cs[j] = c;
    sn[j] = s;
    col[j] = r;
    col[j + 1] = 0.0;
    double gj = gv[j];
    gv[j] = c * gj;
    gv[j + 1] = -s * gj;
    *res_out = fabs(gv[j + 1]);
}

__global__ void k_givens_init(const double* nrm2, double* gv, int m1, double* beta_out, double* inv_beta_out) {
    double b = sqrt(fmax(*nrm2, 0.0));
    for (int i = 0; i < m1; ++i) gv[i] = 0.0;
    gv[0] = b;
    if (beta_out) *beta_out = b;
    *inv_beta_out = b > 0.0 ? 1.0 / b : 0.0;
}

__global__ void k_hess_solve(const double* H, int ldh, const double* gv, int k, double* y) {
    for (int i = k - 1; i >= 0; --i) {
        double s = gv[i];
        for (int l = i + 1; l < k; ++l) s -= H[(long long)l * ldh + i] * y[l];
        double d = H[(long long)i * ldh + i];
        y[i] = d != 0.0 ? s / d : 0.0;
    }
}

inline int blocks_for(long long n) {
    long long b = (n + 255) / 256;
    if (b > 4 * 152 * 4) b = 4 * 152 * 4;
    if (b < 1) b = 1;
    return (int)b;
}

// ---- classical Gram-Schmidt with reorthogonalisation only when needed ------
// st[0] = |w|^2 before projection, st[1] = 1 if a second pass is needed,
// st[2] = |w_perp|^2 used to normalise.

// partial[blk*(k+1) + j] = V_j . w (j < k) and w . w (j == k)
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_mdot_norm(long long n, const T* __restrict__ V, long long ld, int k,
                                                           const T* __restrict__ w, double* __restrict__ partial,
                                                           const double* __restrict__ st) {
    if (st && st[1] == 0.0) return;
    const int K1 = k + 1;
    for (int j0 = 0; j0 < K1; j0 += MDOT_CHUNK) {
        T tacc[MDOT_CHUNK];
#pragma unroll
        for (int q = 0; q < MDOT_CHUNK; ++q) tacc[q] = T(0);
        int nq = min(MDOT_CHUNK, K1 - j0);
        T tacc2[MDOT_CHUNK];
#pragma unroll
        for (int q = 0; q < MDOT_CHUNK; ++q) tacc2[q] = T(0);
        // two elements per trip (i and i + stride) keep twice the loads in flight
        const long long stride = (long long)gridDim.x * blockDim.x;
        long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
        for (; i + stride < n; i += 2 * stride) {
            T wa = w[i], wb = w[i + stride];
#pragma unroll
            for (int q = 0; q < MDOT_CHUNK; ++q) {
                int j = j0 + q;
                if (q < nq) {
                    T va = j < k ? V[(long long)j * ld + i] : wa;
                    T vb = j < k ? V[(long long)j * ld + i + stride] : wb;
                    tacc[q] += va * wa;
                    tacc2[q] += vb * wb;
                }
            }
        }
        if (i < n) {
            T wi = w[i];
#pragma unroll
            for (int q = 0; q < MDOT_CHUNK; ++q) {
                int j = j0 + q;
                if (q < nq) tacc[q] += (j < k ? V[(long long)j * ld + i] : wi) * wi;
            }
        }
#pragma unroll
        for (int q = 0; q < MDOT_CHUNK; ++q) tacc[q] += tacc2[q];
        __shared__ double outv[MDOT_CHUNK];
        block_sum_t<T, MDOT_CHUNK>(tacc, nq, outv);
        if (threadIdx.x < nq) partial[(long long)blockIdx.x * K1 + j0 + threadIdx.x] = outv[threadIdx.x];
        __syncthreads();
    }
}

// after the first pass: dots hk[0..k) and |w|^2 = hk[k]; decide on a second
// pass and clear h2.  The second pass is taken when |w_perp|^2 < |w|^2 / 2
// (the "twice is enough" test).  With the Schur preconditioner the new
// direction lies mostly in the Krylov space already, so in practice the
// second pass runs almost every step; a laxer test cost more outer
// iterations than it saved.
__global__ void k_cgs_state(const double* hk, int k, double* st, double* h2) {
    double nw2 = hk[k], s = 0.0;
    for (int j = 0; j < k; ++j) s += hk[j] * hk[j];
    double nu2 = nw2 - s;
    st[0] = nw2;
    st[1] = (nu2 < 0.5 * nw2) ? 1.0 : 0.0;
    st[2] = nu2 > 0.0 ? nu2 : 0.0;
    const double nu = sqrt(st[2]);
    st[3] = nu > 0.0 ? 1.0 / nu : 0.0;
    for (int j = 0; j < k; ++j) h2[j] = 0.0;
}

// second pass (only when st[1] != 0): w -= V h1
template <typename T>
__global__ void k_cgs_sub(long long n, const T* __restrict__ V, long long ld, int k, const double* __restrict__ h,
                          T* __restrict__ w, const double* __restrict__ st) {
    if (st[1] == 0.0) return;
    __shared__ T hs[128];
    for (int j = threadIdx.x; j < k; j += blockDim.x) hs[j] = (T)h[j];
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        T s = T(0);
        for (int j = 0; j < k; ++j) s += hs[j] * V[(long long)j * ld + i];
        w[i] -= s;
    }
}

// after the second pass's dots: h2 and |w_perp|^2
__global__ void k_cgs_state2(const double* hk2, int k, double* st, double* h2) {
    if (st[1] == 0.0) return;
    double s = 0.0;
    for (int j = 0; j < k; ++j) {
        h2[j] = hk2[j];
        s += hk2[j] * hk2[j];
    }
    double nu2 = hk2[k] - s;
    st[2] = nu2 > 0.0 ? nu2 : 0.0;
    const double nu = sqrt(st[2]);
    st[3] = nu > 0.0 ? 1.0 / nu : 0.0;
}

// V_{k} = (w - sum_j hsel_j V_j) / sqrt(st[2]), hsel = st[1] ? h2 : h1; also an
// optional copy of the first n32 entries in the preconditioner precision
template <typename T, typename T2>
__global__ void k_cgs_normalize(long long n, const T* __restrict__ V, long long ld, int k,
                                const double* __restrict__ h1, const double* __restrict__ h2,
                                const double* __restrict__ st, const T* w, T* vout,  // may alias
                                T2* __restrict__ out2, long long n2) {
    __shared__ double hs[128];
    const double* h = st[1] != 0.0 ? h2 : h1;
    for (int j = threadIdx.x; j < k; j += blockDim.x) hs[j] = h[j];
    __syncthreads();
    const T inv = (T)st[3];  // 1 / sqrt(st[2]), formed by the one-thread state kernel
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (; i + stride < n; i += 2 * stride) {
        T sa = T(0), sb = T(0);
        for (int j = 0; j < k; ++j) {
            T hj = hs[j];
            sa += hj * V[(long long)j * ld + i];
            sb += hj * V[(long long)j * ld + i + stride];
        }
        T va = (w[i] - sa) * inv;
        T vb = (w[i + stride] - sb) * inv;
        vout[i] = va;
        vout[i + stride] = vb;
        if (out2) {
            if (i < n2) out2[i] = (T2)va;
            if (i + stride < n2) out2[i + stride] = (T2)vb;
        }
    }
    if (i < n) {
        T s = T(0);
        for (int j = 0; j < k; ++j) s += hs[j] * V[(long long)j * ld + i];
        T v = (w[i] - s) * inv;
        vout[i] = v;
        if (out2 && i < n2) out2[i] = (T2)v;
    }
}

// y = x * (*inv_norm), plus an optional copy of the first n2 entries
template <typename T, typename T2>
__global__ void k_scale_rsqrt(long long n, const double* __restrict__ inv_norm, const T* __restrict__ x,
                              T* __restrict__ y, T2* __restrict__ out2, long long n2) {
    const T a = (T)*inv_norm;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        T v = a * x[i];
        y[i] = v;
        if (out2 && i < n2) out2[i] = (T2)v;
    }
}


// ---- the outer FGMRES basis in double-float -------------------------------
// V is stored as pairs of floats (value = hi + lo, a 48-bit significand) and
// its Gram-Schmidt dot products and updates run on the FP32 pipe with the
// error-free transformations of Knuth (two-sum) and of the fused multiply-add
// (two-product): on this part the FP64 pipe is ~1/60 of the FP32 pipe, so FP64
// dot and update passes were bound by FP64 arithmetic instead of HBM.  The
// vectors that build the solution (Z, x) stay FP64.
__device__ __forceinline__ dflt df_from(double x) {
    const float h = __double2float_rn(x);
    dflt r;
    r.hi = h;
    r.lo = __double2float_rn(x - (double)h);
    return r;
}
__device__ __forceinline__ double df_to(dflt a) { return (double)a.hi + (double)a.lo; }
// s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// renormalise (|a| >= |b|)
__device__ __forceinline__ dflt quick_two_sum(float a, float b) {
    dflt r;
    r.hi = __fadd_rn(a, b);
    r.lo = __fsub_rn(b, __fsub_rn(r.hi, a));
    return r;
}
// a * b + c
__device__ __forceinline__ dflt df_fma(dflt a, dflt b, dflt c) {
    const float p = __fmul_rn(a.hi, b.hi);
    float pe = __fmaf_rn(a.hi, b.hi, -p);
    pe = __fmaf_rn(a.hi, b.lo, pe);
    pe = __fmaf_rn(a.lo, b.hi, pe);
    float s, e;
    two_sum(p, c.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(pe, c.lo));
    return quick_two_sum(s, e);
}
// a - b
__device__ __forceinline__ dflt df_sub(dflt a, dflt b) {
    float s, e;
    two_sum(a.hi, -b.hi, s, e);
    e = __fadd_rn(e, __fsub_rn(a.lo, b.lo));
    return quick_two_sum(s, e);
}
__device__ __forceinline__ dflt df_zero() {
    dflt r;
    r.hi = 0.f;
    r.lo = 0.f;
    return r;
}

// The basis kernels below work on pairs of entries (one 16-byte load each):
// n2 = number of pairs, ld2 = leading dimension in pairs (the basis is
// allocated with an even length, its pad entry zero).  Loads of the next
// pair are issued before the arithmetic on the current one, and sums over
// basis vectors use independent partial accumulators, so that enough bytes
// are in flight per SM to stream at HBM speed.
__device__ __forceinline__ void ld_pair(const dflt* __restrict__ p, long long q, dflt& a, dflt& b) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p) + q);
    a.hi = v.x;
    a.lo = v.y;
    b.hi = v.z;
    b.lo = v.w;
}
__device__ __forceinline__ void ld_pair_rw(const dflt* p, long long q, dflt& a, dflt& b) {
    const float4 v = reinterpret_cast<const float4*>(p)[q];
    a.hi = v.x;
    a.lo = v.y;
    b.hi = v.z;
    b.lo = v.w;
}
__device__ __forceinline__ void st_pair(dflt* p, long long q, dflt a, dflt b) {
    reinterpret_cast<float4*>(p)[q] = make_float4(a.hi, a.lo, b.hi, b.lo);
}
__device__ __forceinline__ dflt df_add(dflt a, dflt b) {
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    return quick_two_sum(s, e);
}

// w (FP64, n entries) -> double-float in place (same 8 bytes per entry): the
// one pass per Arnoldi step that uses the FP64 pipe
__global__ void k_to_df(long long n, double* w) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const dflt v = df_from(w[i]);
        reinterpret_cast<dflt*>(w)[i] = v;
    }
}

// partial[blk*(k+1) + j] = V_j . w (j < k) and w . w (j == k)
__global__ void __launch_bounds__(RED_THREADS) k_df_mdot_norm(long long n2, const dflt* __restrict__ V, long long ld2,
                                                              int k, const dflt* __restrict__ w,
                                                              double* __restrict__ partial,
                                                              const double* __restrict__ st) {
    if (st && st[1] == 0.0) return;
    const int K1 = k + 1;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int j0 = 0; j0 < K1; j0 += MDOT_CHUNK) {
        const int nv = min(MDOT_CHUNK, k - j0);  // basis vectors in this chunk (may be <= 0)
        const bool with_norm = j0 + MDOT_CHUNK >= K1;
        dflt acc[MDOT_CHUNK];
#pragma unroll
        for (int q = 0; q < MDOT_CHUNK; ++q) acc[q] = df_zero();
        dflt cv[MDOT_CHUNK][2], cw[2];
        long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
        if (p < n2) {
            ld_pair(w, p, cw[0], cw[1]);
#pragma unroll
            for (int q = 0; q < MDOT_CHUNK; ++q)
                if (q < nv) ld_pair(V, (long long)(j0 + q) * ld2 + p, cv[q][0], cv[q][1]);
        }
        while (p < n2) {
            const long long pn = p + stride;
            dflt nv2[MDOT_CHUNK][2], nw[2];
            if (pn < n2) {
                ld_pair(w, pn, nw[0], nw[1]);
#pragma unroll
                for (int q = 0; q < MDOT_CHUNK; ++q)
                    if (q < nv) ld_pair(V, (long long)(j0 + q) * ld2 + pn, nv2[q][0], nv2[q][1]);
            }
#pragma unroll
            for (int q = 0; q < MDOT_CHUNK; ++q) {
                if (q < nv) {
                    acc[q] = df_fma(cv[q][0], cw[0], acc[q]);
                    acc[q] = df_fma(cv[q][1], cw[1], acc[q]);
                } else if (q == nv && with_norm) {
                    acc[q] = df_fma(cw[0], cw[0], acc[q]);
                    acc[q] = df_fma(cw[1], cw[1], acc[q]);
                }
            }
            if (pn < n2) {
                cw[0] = nw[0];
                cw[1] = nw[1];
#pragma unroll
                for (int q = 0; q < MDOT_CHUNK; ++q) {
                    cv[q][0] = nv2[q][0];
                    cv[q][1] = nv2[q][1];
                }
            }
            p = pn;
        }
        double out[MDOT_CHUNK];
#pragma unroll
        for (int q = 0; q < MDOT_CHUNK; ++q) out[q] = df_to(acc[q]);
        __shared__ double outv[MDOT_CHUNK];
        block_sum<MDOT_CHUNK>(out, outv);
        const int nq = min(MDOT_CHUNK, K1 - j0);
        if (threadIdx.x < nq) partial[(long long)blockIdx.x * K1 + j0 + threadIdx.x] = outv[threadIdx.x];
        __syncthreads();
    }
}

// s = sum_{j<k} hs_j V_j at pair q: 8 vectors per trip, loads issued together,
// four independent partial sums
__device__ __forceinline__ void df_combo_pair(const dflt* __restrict__ V, long long ld2, int k, const dflt* hs,
                                              long long q, dflt& s0, dflt& s1) {
    dflt a[4][2];
#pragma unroll
    for (int t = 0; t < 4; ++t) a[t][0] = a[t][1] = df_zero();
    int j = 0;
    for (; j + 8 <= k; j += 8) {
        dflt v[8][2];
#pragma unroll
        for (int u = 0; u < 8; ++u) ld_pair(V, (long long)(j + u) * ld2 + q, v[u][0], v[u][1]);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            a[u & 3][0] = df_fma(hs[j + u], v[u][0], a[u & 3][0]);
            a[u & 3][1] = df_fma(hs[j + u], v[u][1], a[u & 3][1]);
        }
    }
    for (; j < k; ++j) {
        dflt v0, v1;
        ld_pair(V, (long long)j * ld2 + q, v0, v1);
        a[0][0] = df_fma(hs[j], v0, a[0][0]);
        a[0][1] = df_fma(hs[j], v1, a[0][1]);
    }
    s0 = df_add(df_add(a[0][0], a[1][0]), df_add(a[2][0], a[3][0]));
    s1 = df_add(df_add(a[0][1], a[1][1]), df_add(a[2][1], a[3][1]));
}

// second Gram-Schmidt pass (only when st[1] != 0): w <- w - V h
__global__ void __launch_bounds__(RED_THREADS) k_df_sub(long long n2, const dflt* __restrict__ V, long long ld2, int k,
                                                        const double* __restrict__ h, dflt* __restrict__ w,
                                                        const double* __restrict__ st) {
    if (st[1] == 0.0) return;
    __shared__ dflt hs[128];
    for (int j = threadIdx.x; j < k; j += blockDim.x) hs[j] = df_from(h[j]);
    __syncthreads();
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n2;
         p += (long long)gridDim.x * blockDim.x) {
        dflt s0, s1, w0, w1;
        ld_pair_rw(w, p, w0, w1);
        df_combo_pair(V, ld2, k, hs, p, s0, s1);
        st_pair(w, p, df_sub(w0, s0), df_sub(w1, s1));
    }
}

// V_k = (w - V hsel) / sqrt(st[2]) (hsel = st[1] ? h2 : h1); out32[i] (i <
// n32) its float value, out64[i] (from64 <= i < n64) its FP64 value
__global__ void __launch_bounds__(RED_THREADS) k_df_normalize(long long n2, const dflt* __restrict__ V, long long ld2,
                                                              int k, const double* __restrict__ h1,
                                                              const double* __restrict__ h2,
                                                              const double* __restrict__ st,
                                                              const dflt* __restrict__ w, dflt* __restrict__ vout,
                                                              float* __restrict__ out32, long long n32,
                                                              double* __restrict__ out64, long long from64,
                                                              long long n64) {
    __shared__ dflt hs[128];
    const double* h = st[1] != 0.0 ? h2 : h1;
    for (int j = threadIdx.x; j < k; j += blockDim.x) hs[j] = df_from(h[j]);
    __syncthreads();
    const double nu = sqrt(st[2]);
    const dflt inv = df_from(nu > 0.0 ? 1.0 / nu : 0.0);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n2;
         p += (long long)gridDim.x * blockDim.x) {
        dflt s0, s1, w0, w1;
        ld_pair(w, p, w0, w1);
        df_combo_pair(V, ld2, k, hs, p, s0, s1);
        const dflt v0 = df_fma(df_sub(w0, s0), inv, df_zero());
        const dflt v1 = df_fma(df_sub(w1, s1), inv, df_zero());
        st_pair(vout, p, v0, v1);
        const long long i = 2 * p;
        if (out32) {
            if (i < n32) out32[i] = v0.hi;
            if (i + 1 < n32) out32[i + 1] = v1.hi;
        }
        if (out64) {
            if (i >= from64 && i < n64) out64[i] = df_to(v0);
            if (i + 1 >= from64 && i + 1 < n64) out64[i + 1] = df_to(v1);
        }
    }
}

// V_0 = x / sqrt(*nrm2) in double-float (n entries, even), with the same copies
__global__ void k_df_scale(long long n, const double* __restrict__ nrm2, const double* __restrict__ x,
                           dflt* __restrict__ vout, float* __restrict__ out32, long long n32,
                           double* __restrict__ out64, long long from64, long long n64) {
    const double nr = sqrt(fmax(*nrm2, 0.0));
    const dflt a = df_from(nr > 0.0 ? 1.0 / nr : 0.0);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const dflt v = df_fma(df_from(x[i]), a, df_zero());
        vout[i] = v;
        if (out32 && i < n32) out32[i] = v.hi;
        if (out64 && i >= from64 && i < n64) out64[i] = df_to(v);
    }
}

}  // namespace

template <typename T, typename T2>
void cgs_orthonormalize(long long n, const T* V, long long ld, int k, T* w, T* vout, T2* out2, long long n2,
                        double* partial, double* h1, double* h2, double* hk2, double* st, cudaStream_t s) {
    {
        ProfScope ps(KID_MDOT, s, (k + 1.0) * n * sizeof(T));
        k_mdot_norm<T><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, V, ld, k, w, partial, nullptr);
        IBR_CHECK_LAUNCH();
        k_finalize<<<k + 1, RED_THREADS, 0, s>>>(partial, RED_BLOCKS, k + 1, h1);
        IBR_CHECK_LAUNCH();
    }
    {
        ProfScope ps(KID_SMALL, s, 0.0);
        k_cgs_state<<<1, 1, 0, s>>>(h1, k, st, h2);
        IBR_CHECK_LAUNCH();
    }
    {
        // second pass, skipped inside the kernels unless st[1] != 0
        ProfScope ps(KID_UPD_MDOT, s, 0.0);
        k_cgs_sub<T><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, V, ld, k, h1, w, st);
        IBR_CHECK_LAUNCH();
        k_mdot_norm<T><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, V, ld, k, w, partial, st);
        IBR_CHECK_LAUNCH();
        k_finalize<<<k + 1, RED_THREADS, 0, s>>>(partial, RED_BLOCKS, k + 1, hk2);
        IBR_CHECK_LAUNCH();
        k_cgs_state2<<<1, 1, 0, s>>>(hk2, k, st, h2);
        IBR_CHECK_LAUNCH();
    }
    {
        ProfScope ps(KID_UPD_NORM, s, (k + 2.0) * n * sizeof(T) + (out2 ? (double)n2 * sizeof(T2) : 0.0));
        k_cgs_normalize<T, T2><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, V, ld, k, h1, h2, st, w, vout, out2, n2);
        IBR_CHECK_LAUNCH();
    }
}

template <typename T>
void cgs_coeffs_only(long long n, const T* V, long long ld, int k, const T* w, double* partial, double* h1,
                     double* h2, double* st, cudaStream_t s) {
    {
        ProfScope ps(KID_MDOT, s, (k + 1.0) * n * sizeof(T));
        k_mdot_norm<T><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, V, ld, k, w, partial, nullptr);
        IBR_CHECK_LAUNCH();
        k_finalize<<<k + 1, RED_THREADS, 0, s>>>(partial, RED_BLOCKS, k + 1, h1);
        IBR_CHECK_LAUNCH();
    }
    ProfScope ps(KID_SMALL, s, 0.0);
    k_cgs_state<<<1, 1, 0, s>>>(h1, k, st, h2);  // st[2] = max(|w|^2 - |h1|^2, 0), h2 = 0
    IBR_CHECK_LAUNCH();
}

template <typename T, typename T2>
void scale_rsqrt(long long n, const double* inv_norm, const T* x, T* y, T2* out2, long long n2, cudaStream_t s) {
    ProfScope ps(KID_SCALE, s, 2.0 * n * sizeof(T) + (out2 ? (double)n2 * sizeof(T2) : 0.0));
    k_scale_rsqrt<T, T2><<<blocks_for(n), 256, 0, s>>>(n, inv_norm, x, y, out2, n2);
    IBR_CHECK_LAUNCH();
}


void cgs_orthonormalize_df(long long n, long long n_real, const dflt* V, long long ld, int k, double* w, dflt* vout,
                           float* out32, long long n32, double* out64, long long from64, double* partial, double* h1,
                           double* h2, double* hk2, double* st, cudaStream_t s) {
    if ((n & 1) || (ld & 1) || n_real > n)
        throw Error{IBR_EINVAL, "double-float basis: length and leading dimension must be even"};
    dflt* wd = reinterpret_cast<dflt*>(w);
    const long long n2 = n / 2, ld2 = ld / 2;
    {
        ProfScope ps(KID_CONVERT, s, 2.0 * n * 8.0);
        k_to_df<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, w);
        IBR_CHECK_LAUNCH();
    }
    {
        ProfScope ps(KID_MDOT, s, (k + 1.0) * n * 8.0);
        k_df_mdot_norm<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n2, V, ld2, k, wd, partial, nullptr);
        IBR_CHECK_LAUNCH();
        k_finalize<<<k + 1, RED_THREADS, 0, s>>>(partial, RED_BLOCKS, k + 1, h1);
        IBR_CHECK_LAUNCH();
    }
    {
        ProfScope ps(KID_SMALL, s, 0.0);
        k_cgs_state<<<1, 1, 0, s>>>(h1, k, st, h2);
        IBR_CHECK_LAUNCH();
    }
    {
        // second pass, skipped inside the kernels unless st[1] != 0
        ProfScope ps(KID_UPD_MDOT, s, (2.0 * k + 3.0) * n * 8.0);
        k_df_sub<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n2, V, ld2, k, h1, wd, st);
        IBR_CHECK_LAUNCH();
        k_df_mdot_norm<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n2, V, ld2, k, wd, partial, st);
        IBR_CHECK_LAUNCH();
        k_finalize<<<k + 1, RED_THREADS, 0, s>>>(partial, RED_BLOCKS, k + 1, hk2);
        IBR_CHECK_LAUNCH();
        k_cgs_state2<<<1, 1, 0, s>>>(hk2, k, st, h2);
        IBR_CHECK_LAUNCH();
    }
    {
        ProfScope ps(KID_UPD_NORM, s,
                     (k + 2.0) * n * 8.0 + (out32 ? 4.0 * n32 : 0.0) + (out64 ? 8.0 * (n_real - from64) : 0.0));
        k_df_normalize<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n2, V, ld2, k, h1, h2, st, wd, vout, out32, n32, out64,
                                                          from64, n_real);
        IBR_CHECK_LAUNCH();
    }
}

void scale_df(long long n, long long n_real, const double* nrm2, const double* x, dflt* vout, float* out32,
              long long n32, double* out64, long long from64, cudaStream_t s) {
    ProfScope ps(KID_SCALE, s, 16.0 * n);
    k_df_scale<<<blocks_for(n), 256, 0, s>>>(n, nrm2, x, vout, out32, n32, out64, from64, n_real);
    IBR_CHECK_LAUNCH();
}

template void cgs_orthonormalize<double, float>(long long, const double*, long long, int, double*, double*, float*,
                                                long long, double*, double*, double*, double*, double*, cudaStream_t);
template void cgs_orthonormalize<double, double>(long long, const double*, long long, int, double*, double*, double*,
                                                 long long, double*, double*, double*, double*, double*, cudaStream_t);
template void cgs_orthonormalize<float, float>(long long, const float*, long long, int, float*, float*, float*,
                                               long long, double*, double*, double*, double*, double*, cudaStream_t);
template void cgs_coeffs_only<float>(long long, const float*, long long, int, const float*, double*, double*,
                                     double*, double*, cudaStream_t);
template void cgs_coeffs_only<double>(long long, const double*, long long, int, const double*, double*, double*,
                                      double*, double*, cudaStream_t);
template void scale_rsqrt<double, float>(long long, const double*, const double*, double*, float*, long long,
                                         cudaStream_t);
template void scale_rsqrt<double, double>(long long, const double*, const double*, double*, double*, long long,
                                          cudaStream_t);
template void scale_rsqrt<float, float>(long long, const double*, const float*, float*, float*, long long,
                                        cudaStream_t);

namespace {
}  // namespace

template <typename T>
void vec_axpby(long long n, double a, const T* x, double b, T* y, cudaStream_t s) {
    ProfScope ps(KID_AXPBY, s, 3.0 * n * sizeof(T));
    k_axpby<T><<<blocks_for(n), 256, 0, s>>>(n, (T)a, x, (T)b, y);
    IBR_CHECK_LAUNCH();
}
template <typename T>
void vec_scale_copy(long long n, const double* scale_dev, bool invert, const T* x, T* y, cudaStream_t s) {
    ProfScope ps(KID_SCALE, s, 2.0 * n * sizeof(T));
    k_scale_copy<T><<<blocks_for(n), 256, 0, s>>>(n, scale_dev, invert ? 1 : 0, x, y);
    IBR_CHECK_LAUNCH();
}
template <typename Ti, typename To>
void vec_convert(long long n, const Ti* x, To* y, cudaStream_t s) {
    ProfScope ps(KID_CONVERT, s, (double)n * (sizeof(Ti) + sizeof(To)));
    k_convert<Ti, To><<<blocks_for(n), 256, 0, s>>>(n, x, y);
    IBR_CHECK_LAUNCH();
}
template <typename T>
void mdot(long long n, const T* V, long long ld, int k, const T* w, double* partial, double* out, cudaStream_t s) {
    ProfScope ps(KID_MDOT, s, (k + 1.0) * n * sizeof(T));
    k_mdot<T><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, V, ld, k, w, partial);
    IBR_CHECK_LAUNCH();
    k_finalize<<<k, RED_THREADS, 0, s>>>(partial, RED_BLOCKS, k, out);
    IBR_CHECK_LAUNCH();
}
template <typename T>
void update_mdot(long long n, const T* V, long long ld, int k, const double* h, T* w, double* partial, double* out,
                 cudaStream_t s) {
    ProfScope ps(KID_UPD_MDOT, s, (k + 2.0) * n * sizeof(T));
    k_update_mdot<T><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, V, ld, k, h, w, partial);
    IBR_CHECK_LAUNCH();
    k_finalize<<<k, RED_THREADS, 0, s>>>(partial, RED_BLOCKS, k, out);
    IBR_CHECK_LAUNCH();
}
template <typename T>
void update_norm2(long long n, const T* V, long long ld, int k, const double* h, T* w, double* partial, double* out,
                  cudaStream_t s) {
    ProfScope ps(KID_UPD_NORM, s, (k + 2.0) * n * sizeof(T));
    k_update_norm<T><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, V, ld, k, h, w, partial);
    IBR_CHECK_LAUNCH();
    k_finalize<<<1, RED_THREADS, 0, s>>>(partial, RED_BLOCKS, 1, out);
    IBR_CHECK_LAUNCH();
}
template <typename T>
void norm2(long long n, const T* w, double* partial, double* out, cudaStream_t s) {
    ProfScope ps(KID_NORM2, s, (double)n * sizeof(T));
    k_norm2<T><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, w, partial);
    IBR_CHECK_LAUNCH();
    k_finalize<<<1, RED_THREADS, 0, s>>>(partial, RED_BLOCKS, 1, out);
    IBR_CHECK_LAUNCH();
}
template <typename T, typename Tz>
void combine(long long n, const Tz* Z, long long ld, int k, const double* y, T* x, bool accumulate, cudaStream_t s) {
    ProfScope ps(KID_COMBINE, s, (double)n * (k * sizeof(Tz) + (accumulate ? 2 : 1) * sizeof(T)));
    k_combine<T, Tz><<<blocks_for(n), 256, 0, s>>>(n, Z, ld, k, y, x, accumulate ? 1 : 0);
    IBR_CHECK_LAUNCH();
}
template <typename T>
void block_means(long long m, int C, const T* x, double* partial, double* out, cudaStream_t s) {
    ProfScope ps(KID_BLOCK_MEANS, s, (double)m * C * sizeof(T));
    k_block_sums<T><<<RED_BLOCKS, RED_THREADS, 0, s>>>(m, C, x, partial);
    IBR_CHECK_LAUNCH();
    k_finalize<<<C, RED_THREADS, 0, s>>>(partial, RED_BLOCKS, C, out);
    IBR_CHECK_LAUNCH();
    k_scale_vals<<<1, 32, 0, s>>>(C, 1.0 / (double)m, out);
    IBR_CHECK_LAUNCH();
}
template <typename T>
void subtract_means(long long m, int C, T* x, const double* means, cudaStream_t s) {
    ProfScope ps(KID_SUB_MEANS, s, 2.0 * m * C * sizeof(T));
    k_subtract_means<T><<<dim3(blocks_for(m), C), 256, 0, s>>>(m, x, means);
    IBR_CHECK_LAUNCH();
}

void arnoldi_column(double* H, int ldh, const double* h1, const double* h2, const double* nrm2, int j, double* cs,
                    double* sn, double* gv, double* res_out, double* inv_norm_out, cudaStream_t s) {
    ProfScope ps(KID_SMALL, s, 0.0);
    k_arnoldi_column<<<1, 1, 0, s>>>(H, ldh, h1, h2, nrm2, j, cs, sn, gv, res_out, inv_norm_out);
    IBR_CHECK_LAUNCH();
}
void givens_init(const double* nrm2, double* gv, int m1, double* beta_out, double* inv_beta_out, cudaStream_t s) {
    ProfScope ps(KID_SMALL, s, 0.0);
    k_givens_init<<<1, 1, 0, s>>>(nrm2, gv, m1, beta_out, inv_beta_out);
    IBR_CHECK_LAUNCH();
}
void hess_solve(const double* H, int ldh, const double* gv, int k, double* y, cudaStream_t s) {
    ProfScope ps(KID_SMALL, s, 0.0);
    k_hess_solve<<<1, 1, 0, s>>>(H, ldh, gv, k, y);
    IBR_CHECK_LAUNCH();
}

#define IBR_INST(T)                                                                                              \
    template void vec_axpby<T>(long long, double, const T*, double, T*, cudaStream_t);                          \
    template void vec_scale_copy<T>(long long, const double*, bool, const T*, T*, cudaStream_t);                \
    template void mdot<T>(long long, const T*, long long, int, const T*, double*, double*, cudaStream_t);       \
    template void update_mdot<T>(long long, const T*, long long, int, const double*, T*, double*, double*,      \
                                 cudaStream_t);                                                                 \
    template void update_norm2<T>(long long, const T*, long long, int, const double*, T*, double*, double*,     \
                                  cudaStream_t);                                                                \
    template void norm2<T>(long long, const T*, double*, double*, cudaStream_t);                                \
    template void block_means<T>(long long, int, const T*, double*, double*, cudaStream_t);                     \
    template void subtract_means<T>(long long, int, T*, const double*, cudaStream_t);
IBR_INST(double)
IBR_INST(float)
#undef IBR_INST
template void vec_convert<double, float>(long long, const double*, float*, cudaStream_t);
template void vec_convert<float, double>(long long, const float*, double*, cudaStream_t);
template void vec_convert<double, double>(long long, const double*, double*, cudaStream_t);
template void combine<double, double>(long long, const double*, long long, int, const double*, double*, bool,
                                      cudaStream_t);
template void combine<float, float>(long long, const float*, long long, int, const double*, float*, bool,
                                    cudaStream_t);
template void combine<double, float>(long long, const float*, long long, int, const double*, double*, bool,
                                     cudaStream_t);

}  // namespace ibr
