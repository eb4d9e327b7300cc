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


// ---- the Gram-Schmidt passes of the double-float basis, pipelined --------
// One block walks tiles of PG_TP = 256 entry pairs of the system vector.  Its
// producer warp moves the tile's rows (the w row and, per stage, up to PG_CV
// basis rows of 4 KB each) into shared memory with bulk asynchronous copies
// (cp.async.bulk, completion counted in bytes on the stage's "full"
// mbarrier), PG_NST stages ahead of the eight consumer warps, which release a
// stage on its "empty" mbarrier.  Three passes share the pipeline:
//   PG_CONVERT: w (FP64 on entry) is rewritten in place as double-float; the
//               dots V_j . w (j < k) and |w|^2;
//   PG_SUB:     w <- w - V h1 (first sweep over the tile's basis rows), then the
//               dots of the new w (second sweep; the rows come again from the
//               L2); skipped when st[1] == 0 (no second Gram-Schmidt pass);
//   PG_NORM:    V_k = (w - V hsel) / sqrt(st[2]), hsel = st[1] ? h2 : h1, with
//               its FP32 (out32, i < n32) and FP64 (out64, from64 <= i < n64)
//               copies.
// Subtraction: consumer thread t owns pair t of the tile and sums h_j V_j in
// double-float over the basis rows.  Dots: warp g takes row g of each stage
// (basis vectors j = g mod 8), lane l the pairs l + 32 u; each dot is a
// compensated pair (s, c): the product of two double-float entries exact up to
// the lo * lo term (FMA two-product), its high part added to s by Knuth's
// two-sum, every error term to c.  The w tile the dots read is double-
// buffered by tile parity, so one named barrier per tile suffices.  A wait
// that times out sets *err and the block stops.
constexpr int PG_TP = 256;                           // pairs per tile
constexpr int PG_ROW = PG_TP * 16;                   // bytes per row of a tile (4 KB)
constexpr int PG_CV = 8;                             // basis rows per stage
constexpr int PG_NST = 2;                            // stages
constexpr int PG_STAGE = (PG_CV + 1) * PG_ROW;       // w row + PG_CV basis rows
constexpr int PG_CONS = 256;                         // consumer threads (one per pair)
constexpr int PG_THREADS = PG_CONS + 32;             // + the producer warp
constexpr int PG_MAXCH = 16;                         // stages per tile sweep: k <= 128
constexpr int PG_BLOCKS = 2 * 152;                   // two resident blocks per SM
constexpr int PG_SMEM = PG_NST * PG_STAGE            // stages
                        + 3 * PG_ROW                 // w as loaded, w as used (two tiles)
                        + 8 * 16 * 8 + 8 * 8         // per-warp dots, norm
                        + 128 * 8                    // coefficients (double-float)
                        + 2 * PG_NST * 8 + 24;       // mbarriers, issued count, flags
enum { PG_CONVERT = 0, PG_SUB = 1, PG_NORM = 2 };

// (s, c) += v . w over the two entries of a pair (v, w: hi, lo, hi, lo)
__device__ __forceinline__ void dv_acc(const float4 v, const float4 w, float& s, float& c) {
    float p = __fmul_rn(v.x, w.x);
    float e = __fmaf_rn(v.x, w.x, -p);
    e = __fmaf_rn(v.x, w.y, e);
    e = __fmaf_rn(v.y, w.x, e);
    float t, r;
    two_sum(s, p, t, r);
    c = __fadd_rn(c, __fadd_rn(r, e));
    p = __fmul_rn(v.z, w.z);
    e = __fmaf_rn(v.z, w.z, -p);
    e = __fmaf_rn(v.z, w.w, e);
    e = __fmaf_rn(v.w, w.z, e);
    two_sum(t, p, s, r);
    c = __fadd_rn(c, __fadd_rn(r, e));
}
// (s, c) += h x for double-float h and x (the same product and compensation)
__device__ __forceinline__ void dv_axpy(const dflt h, float xh, float xl, float& s, float& c) {
    const float p = __fmul_rn(h.hi, xh);
    float e = __fmaf_rn(h.hi, xh, -p);
    e = __fmaf_rn(h.hi, xl, e);
    e = __fmaf_rn(h.lo, xh, e);
    float t, r;
    two_sum(s, p, t, r);
    s = t;
    c = __fadd_rn(c, __fadd_rn(r, e));
}
// the double-float value of s + c
__device__ __forceinline__ dflt dv_value(float s, float c) {
    float t, r;
    two_sum(s, c, t, r);
    dflt v;
    v.hi = t;
    v.lo = r;
    return v;
}
// (s, c) += (s2, c2)
__device__ __forceinline__ void dv_merge(float& s, float& c, float s2, float c2) {
    float t, r;
    two_sum(s, s2, t, r);
    s = t;
    c = __fadd_rn(c, __fadd_rn(r, c2));
}

__device__ __forceinline__ float4 f4(dflt a, dflt b) { return make_float4(a.hi, a.lo, b.hi, b.lo); }
__device__ __forceinline__ dflt f4a(float4 v) { dflt r; r.hi = v.x; r.lo = v.y; return r; }
__device__ __forceinline__ dflt f4b(float4 v) { dflt r; r.hi = v.z; r.lo = v.w; return r; }

// DF: the basis is double-float (float pairs, arithmetic on the FP32 pipe);
// otherwise FP64 (the same 16-byte pairs, FP64 arithmetic; PG_CONVERT then
// only reads w).
template <int MODE, bool DF>
__global__ void __launch_bounds__(PG_THREADS, 2)
    k_gs_pipe(long long n2, const void* __restrict__ V, long long ld2, int k, void* wv, const double* __restrict__ h1,
              const double* __restrict__ h2, const double* __restrict__ st, double* __restrict__ partial,
              void* __restrict__ vout, float* __restrict__ out32, long long n32, double* __restrict__ out64,
              long long from64, long long n64, int* __restrict__ err) {
    if (MODE == PG_SUB && st[1] == 0.0) return;
    extern __shared__ __align__(128) uint8_t smem[];
    float4* win = reinterpret_cast<float4*>(smem + PG_NST * PG_STAGE);  // w row as loaded
    float4* wuse = win + PG_TP;                                          // [2][PG_TP] w rows the dots use
    double* wred = reinterpret_cast<double*>(wuse + 2 * PG_TP);          // [8][16] per-warp dots
    double* nred = wred + 8 * 16;                                        // [8] norm
    dflt* hs = reinterpret_cast<dflt*>(nred + 8);                        // [128] coefficients (DF)
    double* hd = reinterpret_cast<double*>(hs);                          // [128] coefficients (FP64)
    uint64_t* full = reinterpret_cast<uint64_t*>(hs + 128);
    uint64_t* empty = full + PG_NST;
    long long* issued = reinterpret_cast<long long*>(empty + PG_NST);
    int* fail = reinterpret_cast<int*>(issued + 1);
    int* pdone = fail + 1;
    int* pfail = pdone + 1;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int nch = (k + PG_CV - 1) / PG_CV;
    const long long ntile = (n2 + PG_TP - 1) / PG_TP;
    if (t == 0) {
        *fail = 0;
        *pdone = 0;
        *pfail = 0;
        *issued = 0;
        for (int q = 0; q < PG_NST; ++q) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[q])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;" ::"r"(smem_u32(&empty[q])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (MODE != PG_CONVERT) {
        const double* h = (MODE == PG_NORM && st[1] != 0.0) ? h2 : h1;
        for (int j = t; j < k; j += blockDim.x) {
            if (DF)
                hs[j] = df_from(h[j]);
            else
                hd[j] = h[j];
        }
    }
    __syncthreads();
    const uint32_t sbase = smem_u32(smem);
    if (warp == 8) {
        // producer: one lane issues every copy, in the consumers' order, and
        // leaves the number of items it issued in *issued when it stops
        if (lane == 0) {
            long long it = 0;
            const int sweeps = MODE == PG_SUB ? 2 : 1;
            bool stop = false;
            for (long long tile = blockIdx.x; tile < ntile && !stop; tile += gridDim.x) {
                const long long p0 = tile * PG_TP;
                const uint32_t rb = (uint32_t)(min((long long)PG_TP, n2 - p0) * 16);
                for (int sw = 0; sw < sweeps && !stop; ++sw) {
                    for (int c = 0; c < nch; ++c, ++it) {
                        const int q = (int)(it % PG_NST);
                        if (it >= PG_NST && !mbar_wait(smem_u32(&empty[q]), (uint32_t)((it / PG_NST - 1) & 1))) {
                            // only the consumers write *fail; they learn of this
                            // by their own bounded waits
                            *(volatile int*)pfail = 1;
                            stop = true;
                            break;
                        }
                        if (*(volatile int*)fail) {
                            stop = true;
                            break;
                        }
                        const bool with_w = sw == 0 && c == 0;
                        const int nv = min(PG_CV, k - c * PG_CV);
                        const uint32_t fb = smem_u32(&full[q]);
                        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                                     "r"((with_w ? rb : 0u) + (uint32_t)nv * rb)
                                     : "memory");
                        const uint32_t sq = sbase + q * PG_STAGE;
                        if (with_w) bulk_g2s(sq, reinterpret_cast<const float4*>(wv) + p0, rb, fb);
                        for (int v = 0; v < nv; ++v)
                            bulk_g2s(sq + (v + 1) * PG_ROW,
                                     reinterpret_cast<const float4*>(V) + (long long)(c * PG_CV + v) * ld2 + p0, rb,
                                     fb);
                    }
                }
            }
            *(volatile long long*)issued = it;
            __threadfence_block();
            *(volatile int*)pdone = 1;
        }
        return;
    }
    // consumers (256 threads; named barrier 1 keeps the producer out).  Every
    // consumer thread walks every tile of the block and passes the same named
    // barriers whatever its own waits gave; after a failed wait it waits no
    // more and does no more work.
    // dot accumulators: DF (s, c) float pairs, FP64 in as64
    float as[DF ? PG_MAXCH : 1], ac[DF ? PG_MAXCH : 1];
    double as64[DF ? 1 : PG_MAXCH];
#pragma unroll
    for (int q = 0; q < (DF ? PG_MAXCH : 1); ++q) as[q] = ac[q] = 0.f;
#pragma unroll
    for (int q = 0; q < (DF ? 1 : PG_MAXCH); ++q) as64[q] = 0.0;
    float ns = 0.f, nc = 0.f;
    double nn64 = 0.0;
    dflt inv = df_zero();
    double inv64 = 0.0;
    if (MODE == PG_NORM) {
        // 1 / sqrt(st[2]) from the one-thread state kernel
        if (DF)
            inv = df_from(st[3]);
        else
            inv64 = st[3];
    }
    long long it = 0;
    bool ok = true;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    int par = 0;
    for (long long tile = blockIdx.x; tile < ntile; tile += gridDim.x, par ^= 1) {
        const long long p0 = tile * PG_TP;
        const int np = (int)min((long long)PG_TP, n2 - p0);
        float4* wu = wuse + par * PG_TP;
        if (MODE != PG_CONVERT) {
            // sweep 1: s = V h at pair t (DF: compensated sums), then w - s
            float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f;
            double d0 = 0.0, d1 = 0.0;
            for (int c = 0; c < nch; ++c, ++it) {
                const int q = (int)(it % PG_NST);
                if (ok && !mbar_wait(smem_u32(&full[q]), (uint32_t)((it / PG_NST) & 1))) {
                    ok = false;
                    atomicExch(fail, 1);
                }
                if (!ok) continue;
                const float4* sg = reinterpret_cast<const float4*>(smem + q * PG_STAGE);
                if (c == 0) win[t] = t < np ? sg[t] : z4;
                if (t < np) {
#pragma unroll
                    for (int v = 0; v < PG_CV; ++v) {
                        const int j = c * PG_CV + v;
                        if (j < k) {
                            if constexpr (DF) {
                                const float4 x = sg[(v + 1) * PG_TP + t];
                                const dflt hj = hs[j];
                                dv_axpy(hj, x.x, x.y, s0, c0);
                                dv_axpy(hj, x.z, x.w, s1, c1);
                            } else {
                                const double2 x = reinterpret_cast<const double2*>(sg)[(v + 1) * PG_TP + t];
                                const double hj = hd[j];
                                d0 = fma(hj, x.x, d0);
                                d1 = fma(hj, x.y, d1);
                            }
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[q])) : "memory");
            }
            if (ok) {
                const long long p = p0 + t;
                float4 y = z4;  // w - s (SUB), the new basis entries (NORM)
                float2 y32 = make_float2(0.f, 0.f);
                double y64[2] = {0.0, 0.0};
                if constexpr (DF) {
                    const float4 x = win[t];
                    dflt r0 = df_sub(f4a(x), dv_value(s0, c0)), r1 = df_sub(f4b(x), dv_value(s1, c1));
                    if (MODE == PG_NORM) {
                        r0 = df_fma(r0, inv, df_zero());
                        r1 = df_fma(r1, inv, df_zero());
                        y32 = make_float2(r0.hi, r1.hi);
                        y64[0] = df_to(r0);
                        y64[1] = df_to(r1);
                    }
                    y = f4(r0, r1);
                } else {
                    const double2 x = reinterpret_cast<const double2*>(win)[t];
                    double r0 = x.x - d0, r1 = x.y - d1;
                    if (MODE == PG_NORM) {
                        r0 *= inv64;
                        r1 *= inv64;
                        y32 = make_float2((float)r0, (float)r1);
                        y64[0] = r0;
                        y64[1] = r1;
                    }
                    const double2 yd = make_double2(r0, r1);
                    y = *reinterpret_cast<const float4*>(&yd);
                }
                if (t >= np) y = z4;
                if (MODE == PG_SUB) {
                    wu[t] = y;
                    if (t < np) reinterpret_cast<float4*>(wv)[p] = y;
                } else if (t < np) {
                    reinterpret_cast<float4*>(vout)[p] = y;
                    const long long i = 2 * p;
                    if (out32) {
                        if (i + 1 < n32)
                            *reinterpret_cast<float2*>(out32 + i) = y32;
                        else if (i < n32)
                            out32[i] = y32.x;
                    }
                    if (out64) {
                        if (i >= from64 && i < n64) out64[i] = y64[0];
                        if (i + 1 >= from64 && i + 1 < n64) out64[i + 1] = y64[1];
                    }
                }
            }
            if (MODE == PG_SUB) asm volatile("bar.sync 1, %0;" ::"n"(PG_CONS) : "memory");
        }
        if constexpr (MODE != PG_NORM) {
            // the dot sweep
#pragma unroll
            for (int c = 0; c < PG_MAXCH; ++c) {
                if (c >= nch) break;
                const int q = (int)(it % PG_NST);
                const bool got = ok && mbar_wait(smem_u32(&full[q]), (uint32_t)((it / PG_NST) & 1));
                if (ok && !got) {
                    ok = false;
                    atomicExch(fail, 1);
                }
                ++it;
                const float4* sg = reinterpret_cast<const float4*>(smem + q * PG_STAGE);
                if (MODE == PG_CONVERT && c == 0) {
                    if (got) {
                        float4 y = z4;
                        if (t < np) {
                            if constexpr (DF) {
                                const double2 x = reinterpret_cast<const double2*>(sg)[t];
                                y = f4(df_from(x.x), df_from(x.y));
                                reinterpret_cast<float4*>(wv)[p0 + t] = y;
                            } else {
                                y = sg[t];
                            }
                        }
                        wu[t] = y;
                    }
                    asm volatile("bar.sync 1, %0;" ::"n"(PG_CONS) : "memory");
                }
                if (!got) continue;
                if (c == 0) {
                    if constexpr (DF) {
                        const float4 y = wu[t];
                        dv_acc(y, y, ns, nc);
                    } else {
                        const double2 y = reinterpret_cast<const double2*>(wu)[t];
                        nn64 = fma(y.x, y.x, fma(y.y, y.y, nn64));
                    }
                }
                const int j = c * PG_CV + warp;
                if (j < k) {
                    const float4* row = sg + (warp + 1) * PG_TP;
                    if constexpr (DF) {
                        float s2[2] = {0.f, 0.f}, c2[2] = {0.f, 0.f};
#pragma unroll
                        for (int u = 0; u < PG_TP / 32; ++u) {
                            const int pp = lane + 32 * u;
                            if (pp < np) dv_acc(row[pp], wu[pp], s2[u & 1], c2[u & 1]);
                        }
                        dv_merge(s2[0], c2[0], s2[1], c2[1]);
                        dv_merge(as[c], ac[c], s2[0], c2[0]);
                    } else {
                        const double2* r2 = reinterpret_cast<const double2*>(row);
                        const double2* w2 = reinterpret_cast<const double2*>(wu);
                        double e[2] = {0.0, 0.0};
#pragma unroll
                        for (int u = 0; u < PG_TP / 32; ++u) {
                            const int pp = lane + 32 * u;
                            if (pp < np) {
                                const double2 x = r2[pp], y = w2[pp];
                                e[u & 1] = fma(x.x, y.x, fma(x.y, y.y, e[u & 1]));
                            }
                        }
                        as64[c] += e[0] + e[1];
                    }
                }
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[q])) : "memory");
            }
        }
    }
    asm volatile("bar.sync 1, %0;" ::"n"(PG_CONS) : "memory");
    if (t == 0 && *(volatile int*)pfail) atomicExch(err, 1);
    if (t == 0 && *(volatile int*)fail) {
        // after a time-out: let the producer stop, then wait (bounded) for the
        // copies still in flight into this block's stages before it exits
        atomicExch(err, 1);
        const unsigned long long t0 = global_ns();
        while (!*(volatile int*)pdone && global_ns() - t0 < MBAR_WAIT_LIMIT_NS) {
        }
        const long long ni = *(volatile long long*)issued;
        for (long long x = ni > PG_NST ? ni - PG_NST : 0; x < ni; ++x)
            mbar_wait(smem_u32(&full[x % PG_NST]), (uint32_t)((x / PG_NST) & 1));
    }
    if constexpr (MODE != PG_NORM) {
        // per-warp dots and the norm in FP64, fixed order
#pragma unroll
        for (int c = 0; c < PG_MAXCH; ++c) {
            if (c >= nch) break;
            double x;
            if constexpr (DF)
                x = (double)as[c] + (double)ac[c];
            else
                x = as64[c];
            x = warp_sum(x);
            if (lane == 0) wred[warp * 16 + c] = x;
        }
        const double x = warp_sum(DF ? (double)ns + (double)nc : nn64);
        if (lane == 0) nred[warp] = x;
        asm volatile("bar.sync 1, %0;" ::"n"(PG_CONS) : "memory");
        const int S = k + 1;
        if (t < S) {
            double y = 0.0;
            if (t < k) {
                y = wred[(t % 8) * 16 + t / 8];
            } else {
                for (int g = 0; g < 8; ++g) y += nred[g];
            }
            partial[(long long)blockIdx.x * S + t] = y;
        }
    }
}

// V_0 = x * (*inv_norm) in double-float (n entries, even), with the same copies
__global__ void k_df_scale(long long n, const double* __restrict__ inv_norm, const double* __restrict__ x,
                           dflt* __restrict__ vout, float* __restrict__ out32, long long n32,
                           double* __restrict__ out64, long long from64, long long n64) {
    const dflt a = df_from(*inv_norm);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const dflt v = df_fma(df_from(x[i]), a, df_zero());
        vout[i] = v;
        if (out32 && i < n32) out32[i] = v.hi;
        if (out64 && i >= from64 && i < n64) out64[i] = df_to(v);
    }
}

// ---- modified Gram-Schmidt over the FP64 basis: one pass per basis vector ---
// Step i of MGS subtracts the projection on V_i from w and, in the same pass
// over the entries, forms the dot of the updated w with V_{i+1} (or, after
// the last vector, |w|^2): two FP64 FMAs per entry.  The pass for V_0 only
// forms V_0 . w, the last pass scales w into V_K.  A pass leaves one partial
// sum per block; the next pass reduces them itself, in every block and in a
// fixed order (bitwise the same value everywhere, no separate reduction
// kernel), and block 0 records the coefficient.
constexpr int MG_BLOCKS = 5 * 152;  // five resident blocks of 256 threads per SM (<= 48 registers)

// the sum of the previous pass' partials (fixed order), broadcast to the block
__device__ __forceinline__ double mgs_prev(const double* __restrict__ pin, int nblk, double* sh) {
    double x = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) x += pin[b];
    double v[1] = {x};
    block_sum<1>(v, sh);
    return sh[0];
}

// mode 0: pout = V_0 . w.  mode 1: h = sum(pin), hcol[i] = h (block 0),
// w -= h V_i, pout = V_{i+1} . w (i + 1 < K) or w . w (i + 1 == K).
// n2: entry pairs (n even, a zero pad entry), V_i: rows of ld doubles.
__global__ void __launch_bounds__(RED_THREADS, 5) k_mgs_step(long long n2, const double* __restrict__ Vi,
                                                          const double* __restrict__ Vn, double* __restrict__ w,
                                                          const double* __restrict__ pin, double* __restrict__ pout,
                                                          double* __restrict__ hcol, int mode) {
    pdl_start();
    __shared__ double sh[1];
    double h = 0.0;
    if (mode == 1) {
        h = mgs_prev(pin, gridDim.x, sh);
        if (blockIdx.x == 0 && threadIdx.x == 0) *hcol = h;
    }
    const double2* v2 = reinterpret_cast<const double2*>(Vi);
    const double2* n2p = reinterpret_cast<const double2*>(Vn);  // NULL: the norm of w
    double2* w2 = reinterpret_cast<double2*>(w);
    // two pairs per trip (p and p + stride): their loads are issued together
    double a0 = 0.0, a1 = 0.0, b0 = 0.0, b1 = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (; p + stride < n2; p += 2 * stride) {
        const long long q = p + stride;
        double2 x = w2[p], y = w2[q];
        if (mode == 1) {
            const double2 v = __ldcs(v2 + p), vq = __ldcs(v2 + q);  // last use of V_i in this step
            x.x = fma(-h, v.x, x.x);
            x.y = fma(-h, v.y, x.y);
            y.x = fma(-h, vq.x, y.x);
            y.y = fma(-h, vq.y, y.y);
            w2[p] = x;
            w2[q] = y;
        }
        const double2 u = mode == 0 ? __ldg(v2 + p) : (n2p ? __ldg(n2p + p) : x);
        const double2 uq = mode == 0 ? __ldg(v2 + q) : (n2p ? __ldg(n2p + q) : y);
        a0 = fma(u.x, x.x, a0);
        a1 = fma(u.y, x.y, a1);
        b0 = fma(uq.x, y.x, b0);
        b1 = fma(uq.y, y.y, b1);
    }
    if (p < n2) {
        double2 x = w2[p];
        if (mode == 1) {
            const double2 v = __ldcs(v2 + p);
            x.x = fma(-h, v.x, x.x);
            x.y = fma(-h, v.y, x.y);
            w2[p] = x;
        }
        const double2 u = mode == 0 ? __ldg(v2 + p) : (n2p ? __ldg(n2p + p) : x);
        a0 = fma(u.x, x.x, a0);
        a1 = fma(u.y, x.y, a1);
    }
    double v[1] = {(a0 + a1) + (b0 + b1)};
    block_sum<1>(v, sh);
    if (threadIdx.x == 0) pout[blockIdx.x] = sh[0];
}

// nu^2 = sum(pin) = |w|^2; st[2] = nu^2, st[3] = 1 / nu (block 0);
// V_K = w / nu, out32 (first n32 entries, float) its FP32 copy
__global__ void __launch_bounds__(RED_THREADS, 5) k_mgs_norm(long long n2, const double* __restrict__ w,
                                                          const double* __restrict__ pin, double* __restrict__ st,
                                                          double* __restrict__ vout, float* __restrict__ out32,
                                                          long long n32) {
    pdl_start();
    __shared__ double sh[1];
    __shared__ double inv_s;
    const double nu2 = mgs_prev(pin, gridDim.x, sh);
    if (threadIdx.x == 0) {
        const double nu = sqrt(fmax(nu2, 0.0));
        inv_s = nu > 0.0 ? 1.0 / nu : 0.0;
        if (blockIdx.x == 0) {
            st[0] = nu2;
            st[1] = 0.0;
            st[2] = fmax(nu2, 0.0);
            st[3] = inv_s;
        }
    }
    __syncthreads();
    const double inv = inv_s;
    const double2* w2 = reinterpret_cast<const double2*>(w);
    double2* v2 = reinterpret_cast<double2*>(vout);
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n2;
         p += (long long)gridDim.x * blockDim.x) {
        const double2 x = w2[p];
        const double2 y = make_double2(x.x * inv, x.y * inv);
        v2[p] = y;
        if (out32) {
            const long long i = 2 * p;
            if (i + 1 < n32)
                *reinterpret_cast<float2*>(out32 + i) = make_float2((float)y.x, (float)y.y);
            else if (i < n32)
                out32[i] = (float)y.x;
        }
    }
}

// ---- 16-byte vector variants of the Krylov vector kernels ------------------
// The same operations as k_mdot_norm, k_cgs_sub, k_cgs_normalize, k_norm2,
// k_scale_rsqrt and k_combine over chunks of W = 16 / sizeof(T) entries (one
// 128-bit load per vector and chunk, so four times the bytes in flight of the
// scalar FP32 kernels); the entries past the last whole chunk are handled by
// block 0.  Used when every vector's base is 16-byte aligned (the host checks).
template <typename U, int W>
struct alignas(W * sizeof(U)) PackN {
    U v[W];
};
template <typename T>
using Pk = PackN<T, 16 / (int)sizeof(T)>;

template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_mdot_norm_v(long long n, const T* __restrict__ V, long long ld, int k,
                                                             const T* __restrict__ w, double* __restrict__ partial,
                                                             const double* __restrict__ st) {
    if (st && st[1] == 0.0) return;
    constexpr int W = 16 / (int)sizeof(T);
    const int K1 = k + 1;
    const long long nc = n / W, stride = (long long)gridDim.x * blockDim.x;
    const Pk<T>* w4 = reinterpret_cast<const Pk<T>*>(w);
    for (int j0 = 0; j0 < K1; j0 += MDOT_CHUNK) {
        const int nq = min(MDOT_CHUNK, K1 - j0);
        T tacc[MDOT_CHUNK];
#pragma unroll
        for (int q = 0; q < MDOT_CHUNK; ++q) tacc[q] = T(0);
        for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc; c += stride) {
            const Pk<T> wv = w4[c];
#pragma unroll
            for (int q = 0; q < MDOT_CHUNK; ++q) {
                if (q < nq) {
                    const int j = j0 + q;
                    const Pk<T> vv = j < k ? reinterpret_cast<const Pk<T>*>(V + (long long)j * ld)[c] : wv;
                    T a = tacc[q];
#pragma unroll
                    for (int e = 0; e < W; ++e) a += vv.v[e] * wv.v[e];
                    tacc[q] = a;
                }
            }
        }
        if (blockIdx.x == 0) {
            for (long long i = nc * W + threadIdx.x; i < n; i += blockDim.x) {
                const T wi = w[i];
#pragma unroll
                for (int q = 0; q < MDOT_CHUNK; ++q) {
                    const int j = j0 + q;
                    if (q < nq) tacc[q] += (j < k ? V[(long long)j * ld + i] : wi) * wi;
                }
            }
        }
        __shared__ double outv[MDOT_CHUNK];
        block_sum_t<T, MDOT_CHUNK>(tacc, nq, outv);
        if (threadIdx.x < nq) partial[(long long)blockIdx.x * K1 + j0 + threadIdx.x] = outv[threadIdx.x];
        __syncthreads();
    }
}

// w -= sum_j h_j V_j (only when st[1] != 0)
template <typename T>
__global__ void k_cgs_sub_v(long long n, const T* __restrict__ V, long long ld, int k, const double* __restrict__ h,
                            T* __restrict__ w, const double* __restrict__ st) {
    if (st[1] == 0.0) return;
    constexpr int W = 16 / (int)sizeof(T);
    __shared__ T hs[128];
    for (int j = threadIdx.x; j < k; j += blockDim.x) hs[j] = (T)h[j];
    __syncthreads();
    const long long nc = n / W, stride = (long long)gridDim.x * blockDim.x;
    Pk<T>* w4 = reinterpret_cast<Pk<T>*>(w);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc; c += stride) {
        Pk<T> x = w4[c];
        for (int j = 0; j < k; ++j) {
            const Pk<T> v = reinterpret_cast<const Pk<T>*>(V + (long long)j * ld)[c];
            const T hj = hs[j];
#pragma unroll
            for (int e = 0; e < W; ++e) x.v[e] -= hj * v.v[e];
        }
        w4[c] = x;
    }
    if (blockIdx.x == 0) {
        for (long long i = nc * W + threadIdx.x; i < n; i += blockDim.x) {
            T x = w[i];
            for (int j = 0; j < k; ++j) x -= hs[j] * V[(long long)j * ld + i];
            w[i] = x;
        }
    }
}

// y = s * (x - sum_j h_j V_j) with s = st[3] (k >= 1, h = st[1] ? h2 : h1) or
// s = *inv_norm (k == 0, no V); out2 (first n2 entries) its T2 copy
template <typename T, typename T2>
__global__ void k_scale_sub_v(long long n, const T* __restrict__ V, long long ld, int k, const double* __restrict__ h1,
                              const double* __restrict__ h2, const double* __restrict__ st,
                              const double* __restrict__ inv_norm, const T* x, T* y, T2* __restrict__ out2,
                              long long n2) {
    constexpr int W = 16 / (int)sizeof(T);
    __shared__ T hs[128];
    if (k > 0) {
        const double* h = st[1] != 0.0 ? h2 : h1;
        for (int j = threadIdx.x; j < k; j += blockDim.x) hs[j] = (T)h[j];
    }
    __syncthreads();
    const T sc = (T)(k > 0 ? st[3] : *inv_norm);
    const long long nc = n / W, stride = (long long)gridDim.x * blockDim.x;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc; c += stride) {
        Pk<T> a = reinterpret_cast<const Pk<T>*>(x)[c];
        for (int j = 0; j < k; ++j) {
            const Pk<T> v = reinterpret_cast<const Pk<T>*>(V + (long long)j * ld)[c];
            const T hj = hs[j];
#pragma unroll
            for (int e = 0; e < W; ++e) a.v[e] -= hj * v.v[e];
        }
#pragma unroll
        for (int e = 0; e < W; ++e) a.v[e] *= sc;
        reinterpret_cast<Pk<T>*>(y)[c] = a;
        if (out2) {
            const long long i0 = c * W;
            if (i0 + W <= n2) {
                PackN<T2, W> o;
#pragma unroll
                for (int e = 0; e < W; ++e) o.v[e] = (T2)a.v[e];
                *reinterpret_cast<PackN<T2, W>*>(out2 + i0) = o;
            } else {
#pragma unroll
                for (int e = 0; e < W; ++e)
                    if (i0 + e < n2) out2[i0 + e] = (T2)a.v[e];
            }
        }
    }
    if (blockIdx.x == 0) {
        for (long long i = nc * W + threadIdx.x; i < n; i += blockDim.x) {
            T a = x[i];
            for (int j = 0; j < k; ++j) a -= hs[j] * V[(long long)j * ld + i];
            a *= sc;
            y[i] = a;
            if (out2 && i < n2) out2[i] = (T2)a;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_norm2_v(long long n, const T* __restrict__ w,
                                                         double* __restrict__ partial) {
    constexpr int W = 16 / (int)sizeof(T);
    const long long nc = n / W, stride = (long long)gridDim.x * blockDim.x;
    T acc = T(0);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc; c += stride) {
        const Pk<T> x = reinterpret_cast<const Pk<T>*>(w)[c];
#pragma unroll
        for (int e = 0; e < W; ++e) acc += x.v[e] * x.v[e];
    }
    if (blockIdx.x == 0)
        for (long long i = nc * W + threadIdx.x; i < n; i += blockDim.x) acc += w[i] * w[i];
    T v[1] = {acc};
    __shared__ double o[1];
    block_sum_t<T, 1>(v, 1, o);
    if (threadIdx.x == 0) partial[blockIdx.x] = o[0];
}

// x (+)= sum_j y_j Z_j (T == Tz)
template <typename T>
__global__ void k_combine_v(long long n, const T* __restrict__ Z, long long ld, int k, const double* __restrict__ y,
                            T* __restrict__ x, int accumulate) {
    constexpr int W = 16 / (int)sizeof(T);
    __shared__ T ys[128];
    for (int j = threadIdx.x; j < k; j += blockDim.x) ys[j] = (T)y[j];
    __syncthreads();
    const long long nc = n / W, stride = (long long)gridDim.x * blockDim.x;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc; c += stride) {
        Pk<T> a;
        if (accumulate) {
            a = reinterpret_cast<const Pk<T>*>(x)[c];
        } else {
#pragma unroll
            for (int e = 0; e < W; ++e) a.v[e] = T(0);
        }
        for (int j = 0; j < k; ++j) {
            const Pk<T> z = reinterpret_cast<const Pk<T>*>(Z + (long long)j * ld)[c];
            const T yj = ys[j];
#pragma unroll
            for (int e = 0; e < W; ++e) a.v[e] += yj * z.v[e];
        }
        reinterpret_cast<Pk<T>*>(x)[c] = a;
    }
    if (blockIdx.x == 0) {
        for (long long i = nc * W + threadIdx.x; i < n; i += blockDim.x) {
            T a = accumulate ? x[i] : T(0);
            for (int j = 0; j < k; ++j) a += ys[j] * Z[(long long)j * ld + i];
            x[i] = a;
        }
    }
}

// four entries per thread and trip, 16-byte aligned (one or two 16-byte
// accesses per operand)
template <typename U>
struct alignas(16) Q4 {
    U v[4];
};

template <typename Ti, typename To>
__global__ void k_convert_v(long long n, const Ti* __restrict__ x, To* __restrict__ y) {
    const long long nc = n / 4, stride = (long long)gridDim.x * blockDim.x;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc; c += stride) {
        const Q4<Ti> a = reinterpret_cast<const Q4<Ti>*>(x)[c];
        Q4<To> b;
#pragma unroll
        for (int e = 0; e < 4; ++e) b.v[e] = (To)a.v[e];
        reinterpret_cast<Q4<To>*>(y)[c] = b;
    }
    if (blockIdx.x == 0)
        for (long long i = nc * 4 + threadIdx.x; i < n; i += blockDim.x) y[i] = (To)x[i];
}

// partial[blk*C + c] = this block's sum of component c (m entries each, m % 4 == 0)
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) k_block_sums_v(long long m, int C, const T* __restrict__ x,
                                                              double* __restrict__ partial) {
    const long long mc = m / 4, stride = (long long)gridDim.x * blockDim.x;
    for (int c = 0; c < C; ++c) {
        const Q4<T>* xc = reinterpret_cast<const Q4<T>*>(x + (long long)c * m);
        T t0 = T(0), t1 = T(0);
        for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < mc; q += stride) {
            const Q4<T> a = xc[q];
            t0 += a.v[0] + a.v[2];
            t1 += a.v[1] + a.v[3];
        }
        T v[1] = {t0 + t1};
        __shared__ double o[1];
        block_sum_t<T, 1>(v, 1, o);
        if (threadIdx.x == 0) partial[(long long)blockIdx.x * C + c] = o[0];
    }
}

// component c = blockIdx.y (m % 4 == 0)
template <typename T>
__global__ void k_subtract_means_v(long long m, T* __restrict__ x, const double* __restrict__ means) {
    const T mu = (T)means[blockIdx.y];
    Q4<T>* xc = reinterpret_cast<Q4<T>*>(x + (long long)blockIdx.y * m);
    const long long mc = m / 4;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < mc; q += (long long)gridDim.x * blockDim.x) {
        Q4<T> a = xc[q];
#pragma unroll
        for (int e = 0; e < 4; ++e) a.v[e] -= mu;
        xc[q] = a;
    }
}

inline bool vec16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
template <typename T>
inline bool vec16_basis(const T* V, long long ld) { return vec16(V) && (ld * (long long)sizeof(T)) % 16 == 0; }

}  // namespace

template <typename T, typename T2>
void cgs_orthonormalize(long long n, const T* V, long long ld, int k, T* w, T* vout, T2* out2, long long n2,
                        double* partial, double* h1, double* h2, double* hk2, double* st, cudaStream_t s) {
    // 16-byte vector kernels when every vector is 16-byte aligned
    const bool v = vec16_basis(V, ld) && vec16(w) && vec16(vout) && (!out2 || vec16(out2));
    {
        ProfScope ps(KID_MDOT, s, (k + 1.0) * n * sizeof(T));
        if (v)
            k_mdot_norm_v<T><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, V, ld, k, w, partial, nullptr);
        else
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
        if (v) {
            k_cgs_sub_v<T><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, V, ld, k, h1, w, st);
            IBR_CHECK_LAUNCH();
            k_mdot_norm_v<T><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, V, ld, k, w, partial, st);
        } else {
            k_cgs_sub<T><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, V, ld, k, h1, w, st);
            IBR_CHECK_LAUNCH();
            k_mdot_norm<T><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, V, ld, k, w, partial, st);
        }
        IBR_CHECK_LAUNCH();
        k_finalize<<<k + 1, RED_THREADS, 0, s>>>(partial, RED_BLOCKS, k + 1, hk2);
        IBR_CHECK_LAUNCH();
        k_cgs_state2<<<1, 1, 0, s>>>(hk2, k, st, h2);
        IBR_CHECK_LAUNCH();
    }
    {
        ProfScope ps(KID_UPD_NORM, s, (k + 2.0) * n * sizeof(T) + (out2 ? (double)n2 * sizeof(T2) : 0.0));
        if (v)
            k_scale_sub_v<T, T2><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, V, ld, k, h1, h2, st, nullptr, w, vout, out2,
                                                                    n2);
        else
            k_cgs_normalize<T, T2><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, V, ld, k, h1, h2, st, w, vout, out2, n2);
        IBR_CHECK_LAUNCH();
    }
}

template <typename T>
void cgs_coeffs_only(long long n, const T* V, long long ld, int k, const T* w, double* partial, double* h1,
                     double* h2, double* st, cudaStream_t s) {
    {
        ProfScope ps(KID_MDOT, s, (k + 1.0) * n * sizeof(T));
        if (vec16_basis(V, ld) && vec16(w))
            k_mdot_norm_v<T><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, V, ld, k, w, partial, nullptr);
        else
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
    if (vec16(x) && vec16(y) && (!out2 || vec16(out2)))
        k_scale_sub_v<T, T2><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, (const T*)nullptr, 0, 0, nullptr, nullptr, nullptr,
                                                                inv_norm, x, y, out2, n2);
    else
        k_scale_rsqrt<T, T2><<<blocks_for(n), 256, 0, s>>>(n, inv_norm, x, y, out2, n2);
    IBR_CHECK_LAUNCH();
}


void cgs_orthonormalize_pipe(bool df, long long n, long long n_real, const void* V, long long ld, int k, double* w,
                             void* vout, float* out32, long long n32, double* out64, long long from64,
                             double* partial, double* h1, double* h2, double* hk2, double* st, int* err,
                             cudaStream_t s) {
    if ((n & 1) || (ld & 1) || n_real > n)
        throw Error{IBR_EINVAL, "pipelined Gram-Schmidt: length and leading dimension must be even"};
    if (k < 1 || k > PG_CV * PG_MAXCH) throw Error{IBR_EINVAL, "pipelined Gram-Schmidt: 1 <= k <= 128 required"};
    if ((reinterpret_cast<uintptr_t>(V) | reinterpret_cast<uintptr_t>(w) | reinterpret_cast<uintptr_t>(vout)) & 15)
        throw Error{IBR_EINVAL, "pipelined Gram-Schmidt: V, w and vout must be 16-byte aligned"};
    static PerDeviceOnce once;
    once.run([] {
        const void* f[6] = {(const void*)k_gs_pipe<PG_CONVERT, true>, (const void*)k_gs_pipe<PG_SUB, true>,
                            (const void*)k_gs_pipe<PG_NORM, true>,    (const void*)k_gs_pipe<PG_CONVERT, false>,
                            (const void*)k_gs_pipe<PG_SUB, false>,    (const void*)k_gs_pipe<PG_NORM, false>};
        for (const void* fn : f)
            IBR_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, PG_SMEM));
    });
    const long long n2 = n / 2, ld2 = ld / 2;
    const int grid = (int)std::min<long long>((n2 + PG_TP - 1) / PG_TP, PG_BLOCKS);
    auto conv = df ? k_gs_pipe<PG_CONVERT, true> : k_gs_pipe<PG_CONVERT, false>;
    auto sub = df ? k_gs_pipe<PG_SUB, true> : k_gs_pipe<PG_SUB, false>;
    auto norm = df ? k_gs_pipe<PG_NORM, true> : k_gs_pipe<PG_NORM, false>;
    {
        // first dots and |w|^2 (double-float: w converted in place first)
        ProfScope ps(KID_MDOT, s, (k + (df ? 2.0 : 1.0)) * n * 8.0);
        conv<<<grid, PG_THREADS, PG_SMEM, s>>>(n2, V, ld2, k, w, nullptr, nullptr, nullptr, partial, nullptr, nullptr,
                                               0, nullptr, 0, 0, err);
        IBR_CHECK_LAUNCH();
        k_finalize<<<k + 1, RED_THREADS, 0, s>>>(partial, grid, k + 1, h1);
        IBR_CHECK_LAUNCH();
    }
    {
        ProfScope ps(KID_SMALL, s, 0.0);
        k_cgs_state<<<1, 1, 0, s>>>(h1, k, st, h2);
        IBR_CHECK_LAUNCH();
    }
    {
        // second pass in one kernel, skipped unless st[1] != 0: w -= V h1, then
        // the dots of the new w (the basis rows re-read from the L2)
        ProfScope ps(KID_UPD_MDOT, s, (k + 2.0) * n * 8.0);
        sub<<<grid, PG_THREADS, PG_SMEM, s>>>(n2, V, ld2, k, w, h1, nullptr, st, partial, nullptr, nullptr, 0,
                                              nullptr, 0, 0, err);
        IBR_CHECK_LAUNCH();
        k_finalize<<<k + 1, RED_THREADS, 0, s>>>(partial, grid, k + 1, hk2);
        IBR_CHECK_LAUNCH();
        k_cgs_state2<<<1, 1, 0, s>>>(hk2, k, st, h2);
        IBR_CHECK_LAUNCH();
    }
    {
        ProfScope ps(KID_UPD_NORM, s,
                     (k + 2.0) * n * 8.0 + (out32 ? 4.0 * n32 : 0.0) + (out64 ? 8.0 * (n_real - from64) : 0.0));
        norm<<<grid, PG_THREADS, PG_SMEM, s>>>(n2, V, ld2, k, w, h1, h2, st, nullptr, vout, out32, n32, out64, from64,
                                               n_real, err);
        IBR_CHECK_LAUNCH();
    }
}

void scale_df(long long n, long long n_real, const double* inv_norm, const double* x, dflt* vout, float* out32,
              long long n32, double* out64, long long from64, cudaStream_t s) {
    ProfScope ps(KID_SCALE, s, 16.0 * n);
    k_df_scale<<<blocks_for(n), 256, 0, s>>>(n, inv_norm, x, vout, out32, n32, out64, from64, n_real);
    IBR_CHECK_LAUNCH();
}

void mgs_orthonormalize(long long n, const double* V, long long ld, int k, double* w, double* vout, float* out32,
                        long long n32, double* partial, double* h, double* st, cudaStream_t s) {
    if ((n & 1) || (ld & 1) || k < 1)
        throw Error{IBR_EINVAL, "modified Gram-Schmidt: even length and leading dimension, k >= 1 required"};
    if ((reinterpret_cast<uintptr_t>(V) | reinterpret_cast<uintptr_t>(w) | reinterpret_cast<uintptr_t>(vout)) & 15)
        throw Error{IBR_EINVAL, "modified Gram-Schmidt: V, w and vout must be 16-byte aligned"};
    const long long n2 = n / 2;
    double* pa = partial;
    double* pb = partial + MG_BLOCKS;
    {
        ProfScope ps(KID_MDOT, s, 2.0 * n * 8.0);
        launch_k(k_mgs_step, dim3(MG_BLOCKS), dim3(RED_THREADS), 0, s, n2, V, (const double*)nullptr, w,
                 (const double*)nullptr, pa, (double*)nullptr, 0);
        IBR_CHECK_LAUNCH();
    }
    for (int i = 0; i < k; ++i) {
        // V_i, V_{i+1} (or the norm) and w read, w written
        ProfScope ps(KID_UPD_MDOT, s, (i + 1 < k ? 4.0 : 3.0) * n * 8.0, 4.0 * n);
        const double* Vn = i + 1 < k ? V + (long long)(i + 1) * ld : nullptr;
        launch_k(k_mgs_step, dim3(MG_BLOCKS), dim3(RED_THREADS), 0, s, n2, V + (long long)i * ld, Vn, w,
                 (const double*)pa, pb, h + i, 1);
        IBR_CHECK_LAUNCH();
        std::swap(pa, pb);
    }
    ProfScope ps(KID_UPD_NORM, s, 2.0 * n * 8.0 + (out32 ? 4.0 * n32 : 0.0));
    launch_k(k_mgs_norm, dim3(MG_BLOCKS), dim3(RED_THREADS), 0, s, n2, (const double*)w, (const double*)pa, st, vout,
             out32, n32);
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
    if (vec16(x) && vec16(y))
        k_convert_v<Ti, To><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, x, y);
    else
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
    if (vec16(w))
        k_norm2_v<T><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, w, partial);
    else
        k_norm2<T><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, w, partial);
    IBR_CHECK_LAUNCH();
    k_finalize<<<1, RED_THREADS, 0, s>>>(partial, RED_BLOCKS, 1, out);
    IBR_CHECK_LAUNCH();
}
template <typename T, typename Tz>
void combine(long long n, const Tz* Z, long long ld, int k, const double* y, T* x, bool accumulate, cudaStream_t s) {
    ProfScope ps(KID_COMBINE, s, (double)n * (k * sizeof(Tz) + (accumulate ? 2 : 1) * sizeof(T)));
    if constexpr (std::is_same<T, Tz>::value) {
        if (vec16_basis(Z, ld) && vec16(x) && k <= 128) {
            k_combine_v<T><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, Z, ld, k, y, x, accumulate ? 1 : 0);
            IBR_CHECK_LAUNCH();
            return;
        }
    }
    k_combine<T, Tz><<<blocks_for(n), 256, 0, s>>>(n, Z, ld, k, y, x, accumulate ? 1 : 0);
    IBR_CHECK_LAUNCH();
}
template <typename T>
void block_means(long long m, int C, const T* x, double* partial, double* out, cudaStream_t s) {
    ProfScope ps(KID_BLOCK_MEANS, s, (double)m * C * sizeof(T));
    if (m % 4 == 0 && vec16(x))
        k_block_sums_v<T><<<RED_BLOCKS, RED_THREADS, 0, s>>>(m, C, x, partial);
    else
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
    if (m % 4 == 0 && vec16(x))
        k_subtract_means_v<T><<<dim3(blocks_for(m / 4), C), 256, 0, s>>>(m, x, means);
    else
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
