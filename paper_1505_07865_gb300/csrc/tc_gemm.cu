// Dense products of the approximate-mobility factorisation (Sec. V.C) on the
// 5th-generation tensor cores (sm_103a tcgen05), and the blocked Cholesky /
// triangular inverse / M^-1 = X^T X built from them.
//
// gemm_tf32x3: C = beta C + alpha A B^T for FP32 row-major A [M][K], B [N][K]
// (both K contiguous).  Each operand is split into a TF32 high part and a TF32
// remainder, x = hi + lo, and the three products hi.hi + hi.lo + lo.hi are
// accumulated in FP32 (split-precision TF32, close to FP32 accuracy).  One
// CTA of 128 threads computes a 128 x 128 tile of C: the threads stage 128 x
// 32 slices of A and B (hi and lo) into shared memory in the canonical
// K-major no-swizzle layout (8-row x 16-byte core matrices), double
// buffered; one thread issues tcgen05.mma (kind::tf32, M = N = 128, K = 8)
// into a 128-column TMEM accumulator and commits each slice to an mbarrier;
// the epilogue reads the accumulator with tcgen05.ld.  Every mbarrier wait is
// bounded: on time-out the kernel records an error and stops issuing work.
#include <cstdint>

#include "ibr_internal.cuh"

namespace ibr {
namespace {

constexpr int GT = 128;                   // tile rows / columns
constexpr int GK = 32;                    // K slice per stage
constexpr int SLICE_BYTES = GT * GK * 4;  // one 128 x 32 FP32 slice: 16 KB
constexpr int STAGE_BYTES = 4 * SLICE_BYTES;  // A hi, A lo, B hi, B lo
constexpr int GEMM_SMEM = 2 * STAGE_BYTES + 1024;
constexpr long long WAIT_LIMIT = 1LL << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// shared-memory matrix descriptor: K-major, no swizzle; lbo = byte distance
// of core matrices adjacent along K, sbo = along M/N (8-row groups)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of sm_100-class tensor cores
    return d;                // base offset 0, swizzle mode 0 (none)
}

// instruction descriptor of kind::tf32: D F32, A and B TF32, both K-major,
// N = 128, M = 128
constexpr uint32_t IDESC_TF32_128x128 =
    (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(GT >> 3) << 17) | ((uint32_t)(GT >> 4) << 24);

// byte offset of element (r, k) of a 128 x 32 slice in the canonical layout:
// core matrix (r / 8, k / 4) at ((r / 8) * 8 + k / 4) * 128, row r % 8 at 16
// bytes per row, element k % 4 at 4 bytes
__device__ __forceinline__ uint32_t slice_off(int r, int k) {
    return (uint32_t)((((r >> 3) << 3) + (k >> 2)) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(IDESC_TF32_128x128), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

// bounded wait for the phase with the given parity; false on time-out
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (long long it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// load a 128 x 32 slice of a row-major FP32 matrix (rows r0.., columns k0..)
// and store its TF32 high and low parts; thread t handles 8 of the 1024
// 16-byte chunks: chunk q -> row (q & 7) + 8 (q >> 6), chunk column (q >> 3) & 7
// (8 consecutive threads: 8 rows of one chunk column, conflict-free stores)
__device__ __forceinline__ void stage_slice(const float* __restrict__ X, int ld, int r0, int k0, uint8_t* hi,
                                            uint8_t* lo) {
    const int t = threadIdx.x;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int q = i * GT + t;
        const int r = (q & 7) + 8 * (q >> 6);
        const int c = (q >> 3) & 7;
        const float4 v = *reinterpret_cast<const float4*>(X + (long long)(r0 + r) * ld + k0 + 4 * c);
        float4 h, l;
        h.x = tf32_round(v.x);
        h.y = tf32_round(v.y);
        h.z = tf32_round(v.z);
        h.w = tf32_round(v.w);
        l.x = tf32_round(v.x - h.x);
        l.y = tf32_round(v.y - h.y);
        l.z = tf32_round(v.z - h.z);
        l.w = tf32_round(v.w - h.w);
        const uint32_t off = slice_off(r, 4 * c);
        *reinterpret_cast<float4*>(hi + off) = h;
        *reinterpret_cast<float4*>(lo + off) = l;
    }
}

// C may overlap A (the in-place panel product): a CTA reads all of its A rows
// before it writes its C tile, and no other CTA reads them
__global__ void __launch_bounds__(GT) k_gemm_tf32x3(int K, const float* A, int lda,
                                                    const float* __restrict__ B, int ldb, float* C, int ldc,
                                                    float alpha, float beta, int lower_only, int* __restrict__ err) {
    const int tm = blockIdx.y, tn = blockIdx.x;
    if (lower_only && tn > tm) return;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* stage0 = smem;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * STAGE_BYTES);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 2 * STAGE_BYTES + 64);
    const int t = threadIdx.x, warp = t >> 5;
    if (t == 0) {
        for (int s = 0; s < 2; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[s])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(GT));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const int m0 = tm * GT, n0 = tn * GT;
    const int nk = K / GK;
    bool ok = true;
    for (int kc = 0; kc < nk; ++kc) {
        const int s = kc & 1;
        uint8_t* st = stage0 + s * STAGE_BYTES;
        // the MMAs that last read this stage (slice kc - 2) must be done; the
        // decision to go on is the same for every thread of the CTA
        if (kc >= 2) ok = mbar_wait(smem_u32(&mbar[s]), ((kc - 2) >> 1) & 1);
        if (!__syncthreads_and(ok ? 1 : 0)) {
            ok = false;
            break;
        }
        stage_slice(A, lda, m0, kc * GK, st, st + SLICE_BYTES);
        stage_slice(B, ldb, n0, kc * GK, st + 2 * SLICE_BYTES, st + 3 * SLICE_BYTES);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a_hi = smem_u32(st), a_lo = a_hi + SLICE_BYTES;
            const uint32_t b_hi = a_hi + 2 * SLICE_BYTES, b_lo = a_hi + 3 * SLICE_BYTES;
#pragma unroll
            for (int j = 0; j < GK / 8; ++j) {
                // K = 8 per instruction: two core matrices along K (256 bytes)
                const uint32_t o = j * 256;
                const uint64_t dah = smem_desc(a_hi + o, 128, 1024), dal = smem_desc(a_lo + o, 128, 1024);
                const uint64_t dbh = smem_desc(b_hi + o, 128, 1024), dbl = smem_desc(b_lo + o, 128, 1024);
                mma_tf32(tmem, dah, dbh, (kc > 0 || j > 0) ? 1u : 0u);
                mma_tf32(tmem, dah, dbl, 1u);
                mma_tf32(tmem, dal, dbh, 1u);
            }
            mma_commit(smem_u32(&mbar[s]));
        }
    }
    // the last commit covers every MMA issued before it
    if (ok && nk > 0) ok = mbar_wait(smem_u32(&mbar[(nk - 1) & 1]), ((nk - 1) >> 1) & 1);
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
    if (!ok && t == 0) atomicExch(err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        // warp w reads TMEM lanes 32w..32w+31 = rows m0 + 32w + lane
        const int row = m0 + warp * 32 + (t & 31);
        float* Cr = C + (long long)row * ldc + n0;
#pragma unroll 1
        for (int c0 = 0; c0 < GT; c0 += 8) {
            uint32_t v[8];
            const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const float r = alpha * __uint_as_float(v[e]);
                Cr[c0 + e] = beta == 0.0f ? r : r + beta * Cr[c0 + e];
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(GT));
}

// ---------------------------------------------------------------------------
// blocked factorisation pieces (P = 128 blocks, CUDA cores)

// Cholesky of the P x P diagonal block at (k, k) of A (ld) in shared memory:
// A_kk = L L^T, L written back (lower, zeros above), Dinv = L^-1 (lower, P x
// P row-major).  info = global pivot index + 1 if a pivot <= min_pivot.
__global__ void __launch_bounds__(GT) k_diag_block(float* __restrict__ A, int ld, int k, float* __restrict__ Dinv,
                                                   int* __restrict__ info, float min_pivot) {
    extern __shared__ __align__(16) float sm[];
    float* L = sm;                   // [GT][GT + 1]
    float* X = sm + GT * (GT + 1);   // [GT][GT + 1]
    const int t = threadIdx.x;
    float* Akk = A + (long long)k * GT * ld + (long long)k * GT;
    for (int r = 0; r < GT; ++r) L[r * (GT + 1) + t] = Akk[(long long)r * ld + t];
    __syncthreads();
    for (int j = 0; j < GT; ++j) {
        if (t == 0) {
            float dj = L[j * (GT + 1) + j];
            if (!(dj > min_pivot)) {
                if (*info == 0) *info = k * GT + j + 1;
                dj = fmaxf(fabsf(dj), min_pivot > 0.f ? min_pivot : 1e-30f);
            }
            L[j * (GT + 1) + j] = sqrtf(dj);
        }
        __syncthreads();
        const float djj = L[j * (GT + 1) + j];
        if (t > j) L[t * (GT + 1) + j] /= djj;
        __syncthreads();
        // trailing update of column t (rows >= t) by column j
        if (t > j) {
            const float ltj = L[t * (GT + 1) + j];
            for (int i = t; i < GT; ++i) L[i * (GT + 1) + t] -= L[i * (GT + 1) + j] * ltj;
        }
        __syncthreads();
    }
    // X = L^-1: thread t solves L x = e_t (column t of X) by forward substitution
    for (int r = 0; r < GT; ++r) {
        float s = (r == t) ? 1.0f : 0.0f;
        for (int q = t; q < r; ++q) s -= L[r * (GT + 1) + q] * X[q * (GT + 1) + t];
        X[r * (GT + 1) + t] = (r >= t) ? s / L[r * (GT + 1) + r] : 0.0f;
    }
    __syncthreads();
    for (int r = 0; r < GT; ++r) {
        Akk[(long long)r * ld + t] = (t <= r) ? L[r * (GT + 1) + t] : 0.0f;
        Dinv[r * GT + t] = X[r * (GT + 1) + t];
    }
}

// XT block (i, i) = Dinv_i^T
__global__ void k_put_diag_t(float* __restrict__ XT, int ld, int i, const float* __restrict__ Dinv) {
    const int t = threadIdx.x;
    for (int r = 0; r < GT; ++r) XT[(long long)(i * GT + r) * ld + i * GT + t] = Dinv[t * GT + r];
}

// padded copy: P = [[M, 0], [0, pad I]] (n x n inside np x np)
__global__ void k_pad_in(int n, int np, const float* __restrict__ M, float* __restrict__ P, float pad) {
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= (long long)np * np) return;
    const int r = (int)(id / np), c = (int)(id % np);
    P[id] = (r < n && c < n) ? M[(long long)r * n + c] : (r == c ? pad : 0.0f);
}

// M = the n x n corner of the symmetric result whose lower triangle is in P
__global__ void k_sym_out(int n, int np, const float* __restrict__ P, float* __restrict__ M) {
    const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (id >= (long long)n * n) return;
    const int r = (int)(id / n), c = (int)(id % n);
    M[id] = c <= r ? P[(long long)r * np + c] : P[(long long)c * np + r];
}

void set_attributes() {
    static const bool done = [] {
        IBR_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tf32x3, cudaFuncAttributeMaxDynamicSharedMemorySize, GEMM_SMEM));
        IBR_CUDA_TRY(cudaFuncSetAttribute(k_diag_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)(2 * GT * (GT + 1) * sizeof(float))));
        return true;
    }();
    (void)done;
}

}  // namespace

void gemm_tf32x3(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc, float alpha,
                 float beta, bool lower_only, int* err_dev, cudaStream_t s) {
    if (M % GT || N % GT || K % GK || lda % 4 || ldb % 4)
        throw Error{IBR_EINVAL, "gemm_tf32x3: M, N must be multiples of 128, K of 32, lda and ldb of 4"};
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15)
        throw Error{IBR_EINVAL, "gemm_tf32x3: A and B must be 16-byte aligned"};
    if (M == 0 || N == 0) return;
    set_attributes();
    ProfScope ps(KID_TC_GEMM, s, 4.0 * ((double)M * K + (double)N * K + 2.0 * M * N));
    dim3 grid(N / GT, M / GT);
    k_gemm_tf32x3<<<grid, GT, GEMM_SMEM, s>>>(K, A, lda, B, ldb, C, ldc, alpha, beta, lower_only ? 1 : 0, err_dev);
    IBR_CHECK_LAUNCH();
}

// M (n x n SPD, FP32, row-major) -> M^-1 on the tensor cores: padded to a
// multiple of 128 with an identity block, blocked right-looking Cholesky
// (diagonal blocks on CUDA cores, panel A_ik L_kk^-T and trailing update
// A_ij -= L_ik L_jk^T as tensor-core products), X^T = (L^-1)^T block column by
// block column (U = X^T[0:i,0:i] L_i,0:i^T, X^T[0:i, i] = -U L_ii^-T), then
// M^-1 = X^T (X^T)^T (lower tiles) and the symmetric n x n corner.
void spd_inverse_tc(int n, float* M, int* info_dev, double min_pivot, double pad, int* err_dev, cudaStream_t s) {
    set_attributes();
    const int np = (n + GT - 1) / GT * GT;
    const int nb = np / GT;
    float *P = nullptr, *XT = nullptr, *U = nullptr, *Dinv = nullptr;
    IBR_CUDA_TRY(cudaMallocAsync(&P, (size_t)np * np * sizeof(float), s));
    IBR_CUDA_TRY(cudaMallocAsync(&XT, (size_t)np * np * sizeof(float), s));
    IBR_CUDA_TRY(cudaMallocAsync(&U, (size_t)np * GT * sizeof(float), s));
    IBR_CUDA_TRY(cudaMallocAsync(&Dinv, (size_t)nb * GT * GT * sizeof(float), s));
    const long long np2 = (long long)np * np;
    {
        ProfScope ps(KID_SPD_INV, s, 4.0 * ((double)n * n + (double)np2));
        k_pad_in<<<grid_1d(np2, 256), 256, 0, s>>>(n, np, M, P, (float)pad);
        IBR_CHECK_LAUNCH();
    }
    for (int k = 0; k < nb; ++k) {
        {
            ProfScope ps(KID_SPD_INV, s, 4.0 * 3 * GT * GT);
            k_diag_block<<<1, GT, 2 * GT * (GT + 1) * sizeof(float), s>>>(P, np, k, Dinv + (long long)k * GT * GT,
                                                                          info_dev, (float)min_pivot);
            IBR_CHECK_LAUNCH();
        }
        const int rest = np - (k + 1) * GT;
        if (rest > 0) {
            float* pan = P + (long long)(k + 1) * GT * np + (long long)k * GT;
            gemm_tf32x3(rest, GT, GT, pan, np, Dinv + (long long)k * GT * GT, GT, pan, np, 1.f, 0.f, false, err_dev, s);
            float* tr = P + (long long)(k + 1) * GT * np + (long long)(k + 1) * GT;
            gemm_tf32x3(rest, rest, GT, pan, np, pan, np, tr, np, -1.f, 1.f, true, err_dev, s);
        }
    }
    IBR_CUDA_TRY(cudaMemsetAsync(XT, 0, (size_t)np2 * sizeof(float), s));
    for (int i = 0; i < nb; ++i) {
        {
            ProfScope ps(KID_SPD_INV, s, 4.0 * 2 * GT * GT);
            k_put_diag_t<<<1, GT, 0, s>>>(XT, np, i, Dinv + (long long)i * GT * GT);
            IBR_CHECK_LAUNCH();
        }
        if (i > 0) {
            const int m = i * GT;
            gemm_tf32x3(m, GT, m, XT, np, P + (long long)i * GT * np, np, U, GT, 1.f, 0.f, false, err_dev, s);
            gemm_tf32x3(m, GT, GT, U, GT, Dinv + (long long)i * GT * GT, GT, XT + (long long)i * GT, np, -1.f, 0.f,
                        false, err_dev, s);
        }
    }
    gemm_tf32x3(np, np, np, XT, np, XT, np, P, np, 1.f, 0.f, true, err_dev, s);
    {
        ProfScope ps(KID_SPD_INV, s, 4.0 * 2.0 * n * n);
        k_sym_out<<<grid_1d((long long)n * n, 256), 256, 0, s>>>(n, np, P, M);
        IBR_CHECK_LAUNCH();
    }
    IBR_CUDA_TRY(cudaFreeAsync(P, s));
    IBR_CUDA_TRY(cudaFreeAsync(XT, s));
    IBR_CUDA_TRY(cudaFreeAsync(U, s));
    IBR_CUDA_TRY(cudaFreeAsync(Dinv, s));
}

}  // namespace ibr
