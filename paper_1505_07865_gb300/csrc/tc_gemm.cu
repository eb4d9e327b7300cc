// Dense products of the approximate-mobility factorisation (Sec. V.C) on the
// 5th-generation tensor cores (sm_103a tcgen05), and the blocked Cholesky /
// triangular inverse / M^-1 = X^T X built from them.
//
// gemm_tf32x3: C = beta C + alpha A B^T for FP32 row-major A [M][K], B [N][K]
// (both K contiguous).  Each operand is split into a TF32 high part and a TF32
// remainder, x = hi + lo, and the three products hi.hi + hi.lo + lo.hi are
// accumulated in FP32 (split-precision TF32, close to FP32 accuracy).  A pack
// pass writes the hi and lo parts in 128 x 32 slices already laid out as the
// tensor cores read them from shared memory (canonical K-major, no swizzle:
// 8-row x 16-byte core matrices); one CTA per 128 x 128 tile of C then runs a
// producer / consumer pipeline over three shared-memory stages: one thread
// moves slices with bulk asynchronous copies (cp.async.bulk, completion counted
// on an mbarrier), one thread issues tcgen05.mma (kind::tf32, M = N = 128,
// K = 8) into a 128-column TMEM accumulator and commits each slice back to the
// producer; the epilogue reads the accumulator with tcgen05.ld.  Every
// mbarrier wait is bounded: on time-out the kernel records an error and stops
// issuing work.
#include <cstdint>

#include "ibr_internal.cuh"

namespace ibr {
namespace {

constexpr int GT = 128;                   // tile rows / columns
constexpr int GK = 32;                    // K slice per stage
constexpr int NSTAGE = 3;                 // slices in flight
constexpr int SLICE_BYTES = GT * GK * 4;  // one 128 x 32 FP32 slice: 16 KB
constexpr int STAGE_BYTES = 4 * SLICE_BYTES;  // A hi, A lo, B hi, B lo
constexpr int GEMM_SMEM = NSTAGE * STAGE_BYTES + 256;


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

// Operand packing: the TF32 high and low parts of a row-major FP32 matrix
// (rows a multiple of 128, K a multiple of 32), each 128 x 32 slice stored as
// one contiguous 16 KB block already in the canonical shared-memory layout
// (slice (mt, kt) at ((mt * K / 32) + kt) * 4096 floats), so that the product
// kernel moves whole slices with one bulk copy each.
__global__ void k_pack_tf32(const float* __restrict__ X, int ld, int rows, int K, float* __restrict__ hi,
                            float* __restrict__ lo) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;  // 16-byte chunk
    const int kq = K / 4;
    if (q >= (long long)rows * kq) return;
    const int r = (int)(q / kq), c4 = (int)(q % kq);
    const float4 v = *reinterpret_cast<const float4*>(X + (long long)r * ld + 4 * c4);
    float4 h, l;
    h.x = tf32_round(v.x);
    h.y = tf32_round(v.y);
    h.z = tf32_round(v.z);
    h.w = tf32_round(v.w);
    l.x = tf32_round(v.x - h.x);
    l.y = tf32_round(v.y - h.y);
    l.z = tf32_round(v.z - h.z);
    l.w = tf32_round(v.w - h.w);
    const long long slice = (long long)(r / GT) * (K / GK) + (4 * c4) / GK;
    const long long off = slice * (GT * GK) + slice_off(r % GT, (4 * c4) % GK) / 4;
    *reinterpret_cast<float4*>(hi + off) = h;
    *reinterpret_cast<float4*>(lo + off) = l;
}


// One CTA per 128 x 128 tile of C.  Thread 32 (producer) fills a free stage
// with the four slices of K slice kc (bulk copies, completion counted in
// bytes on full[s]); thread 0 (consumer) waits for full[s], issues the 12
// MMAs of the slice and commits them to empty[s]; after the last slice a
// commit to done releases the epilogue (all four warps read their TMEM lane
// quarter).  Pa*/Pb*: packed operands; mt, nt: tile row / column.
__global__ void __launch_bounds__(GT) k_gemm_tf32x3(int K, const float* __restrict__ Pah,
                                                    const float* __restrict__ Pal, const float* __restrict__ Pbh,
                                                    const float* __restrict__ Pbl, float* C, int ldc, float alpha,
                                                    float beta, int lower_only, int* __restrict__ err) {
    const int tm = blockIdx.y, tn = blockIdx.x;
    if (lower_only && tn > tm) return;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + NSTAGE * STAGE_BYTES);
    uint64_t* empty = full + NSTAGE;
    uint64_t* done = empty + NSTAGE;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    __shared__ int fail;
    const int t = threadIdx.x, warp = t >> 5;
    if (t == 0) {
        fail = 0;
        for (int s = 0; s < NSTAGE; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(done)));
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
    const int nk = K / GK;
    const long long a0 = (long long)tm * nk * (GT * GK), b0 = (long long)tn * nk * (GT * GK);
    const uint32_t base = smem_u32(smem);
    if (t == 32) {
        // producer
        for (int kc = 0; kc < nk; ++kc) {
            const int s = kc % NSTAGE;
            if (kc >= NSTAGE && !mbar_wait(smem_u32(&empty[s]), (uint32_t)((kc / NSTAGE - 1) & 1))) {
                fail = 1;
                break;
            }
            if (*(volatile int*)&fail) break;
            const uint32_t fb = smem_u32(&full[s]);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(STAGE_BYTES)
                         : "memory");
            const uint32_t st = base + s * STAGE_BYTES;
            const long long so = (long long)kc * (GT * GK);
            bulk_g2s(st, Pah + a0 + so, SLICE_BYTES, fb);
            bulk_g2s(st + SLICE_BYTES, Pal + a0 + so, SLICE_BYTES, fb);
            bulk_g2s(st + 2 * SLICE_BYTES, Pbh + b0 + so, SLICE_BYTES, fb);
            bulk_g2s(st + 3 * SLICE_BYTES, Pbl + b0 + so, SLICE_BYTES, fb);
        }
    } else if (t == 0) {
        // consumer: the MMA issuer
        for (int kc = 0; kc < nk; ++kc) {
            const int s = kc % NSTAGE;
            if (!mbar_wait(smem_u32(&full[s]), (uint32_t)((kc / NSTAGE) & 1))) {
                fail = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a_hi = base + s * STAGE_BYTES, a_lo = a_hi + SLICE_BYTES;
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
            mma_commit(smem_u32(&empty[s]));
        }
        mma_commit(smem_u32(done));  // every MMA issued above
    }
    __syncthreads();
    // the accumulator is final once done completes (bounded wait)
    bool ok = !fail && nk > 0;
    if (ok) ok = mbar_wait(smem_u32(done), 0);
    ok = __syncthreads_and(ok ? 1 : 0) != 0;
    if (!ok && t == 0) atomicExch(err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        // warp w reads TMEM lanes 32w..32w+31 = rows 32w + lane of the tile
        const int row = tm * GT + warp * 32 + (t & 31);
        float* Cr = C + (long long)row * ldc + tn * GT;
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
// Blocked by 32 (P = 4 x 32): warp 0 factors and inverts each 32 x 32
// diagonal block in registers (lane i holds row i; values move by shuffles);
// the 16 warps then form the panel below it (A_ik W_k^T, W_k = L_kk^-1) and the
// trailing update; finally X = L^-1 block row by block row,
// X_ik = -W_i sum_{j=k}^{i-1} L_ij X_jk.
constexpr int DB_THREADS = 512;
constexpr int DB_LD = GT + 1;
constexpr int DB_SMEM = (2 * GT * DB_LD + 4 * 32 * 33 + 32 * 97) * (int)sizeof(float);

__global__ void __launch_bounds__(DB_THREADS) k_diag_block(float* __restrict__ A, int ld, int k,
                                                           float* __restrict__ Dinv, int* __restrict__ info,
                                                           float min_pivot) {
    extern __shared__ __align__(16) float sm[];
    float* L = sm;                    // [GT][DB_LD]
    float* X = L + GT * DB_LD;        // [GT][DB_LD]
    float* W = X + GT * DB_LD;        // [4][32][33]: inverses of the 32 x 32 diagonal blocks
    float* T = W + 4 * 32 * 33;       // [32][97]
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const unsigned FULL = 0xffffffffu;
    float* Akk = A + (long long)k * GT * ld + (long long)k * GT;
    for (int e = t; e < GT * GT; e += DB_THREADS) {
        const int r = e >> 7, c = e & (GT - 1);
        L[r * DB_LD + c] = Akk[(long long)r * ld + c];
        X[r * DB_LD + c] = 0.0f;
    }
    __syncthreads();
    const float floor_piv = min_pivot > 0.f ? min_pivot : 1e-30f;
    for (int kb = 0; kb < 4; ++kb) {
        const int o = kb * 32;
        if (warp == 0) {
            // lane i holds row i; the finished column j goes through shared
            // memory (col), so that the updates of the later columns read it
            // as independent broadcast loads instead of a chain of shuffles
            float r[32], x[32];
            float* col = T;
#pragma unroll
            for (int c = 0; c < 32; ++c) r[c] = L[(o + lane) * DB_LD + o + c];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                float djj = __shfl_sync(FULL, r[j], j);
                if (!(djj > min_pivot)) {
                    if (lane == j && *info == 0) *info = k * GT + o + j + 1;
                    djj = fmaxf(fabsf(djj), floor_piv);
                }
                const float sq = sqrtf(djj);
                r[j] = lane == j ? sq : (lane > j ? r[j] / sq : r[j]);
                col[lane] = r[j];
                __syncwarp();
#pragma unroll
                for (int c = j + 1; c < 32; ++c)
                    if (lane >= c) r[c] -= r[j] * col[c];
                __syncwarp();
            }
#pragma unroll
            for (int c = 0; c < 32; ++c) L[(o + lane) * DB_LD + o + c] = c <= lane ? r[c] : 0.0f;
            __syncwarp();
            // column `lane` of the inverse by forward substitution; row rr of the
            // factor is read from shared memory (broadcast), two partial sums
#pragma unroll
            for (int rr = 0; rr < 32; ++rr) {
                const float* Lr = L + (o + rr) * DB_LD + o;
                float s0 = lane == rr ? 1.0f : 0.0f, s1 = 0.0f;
#pragma unroll
                for (int q = 0; q < rr; ++q) {
                    if (q & 1)
                        s1 -= Lr[q] * x[q];
                    else
                        s0 -= Lr[q] * x[q];
                }
                x[rr] = rr >= lane ? (s0 + s1) / Lr[rr] : 0.0f;
            }
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                W[(kb * 32 + c) * 33 + lane] = x[c];
                X[(o + c) * DB_LD + o + lane] = x[c];
            }
        }
        __syncthreads();
        const int R0 = o + 32;
        if (R0 < GT) {
            // panel: L[r][o + c] = sum_{q <= c} A[r][o + q] W_kb[c][q], rows r >= R0
            float pv[(GT - 32) * 32 / DB_THREADS];
            const int ne = (GT - R0) * 32;
#pragma unroll
            for (int u = 0; u < (GT - 32) * 32 / DB_THREADS; ++u) {
                const int e = t + u * DB_THREADS;
                float acc = 0.0f;
                if (e < ne) {
                    const int r = R0 + (e >> 5), c = e & 31;
                    for (int q = 0; q <= c; ++q) acc += L[r * DB_LD + o + q] * W[(kb * 32 + c) * 33 + q];
                }
                pv[u] = acc;
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < (GT - 32) * 32 / DB_THREADS; ++u) {
                const int e = t + u * DB_THREADS;
                if (e < ne) L[(R0 + (e >> 5)) * DB_LD + o + (e & 31)] = pv[u];
            }
            __syncthreads();
            // trailing update of the lower part at rows, columns >= R0: thread
            // (lane, warp) owns rows warp + 16 a and columns lane + 32 b, an
            // 8 x 4 register tile, so each panel entry loaded from shared
            // memory serves four (row) or eight (column) products
            const int tx = lane, ty = warp;
            float acc[GT / 16][GT / 32];
#pragma unroll
            for (int a = 0; a < GT / 16; ++a)
#pragma unroll
                for (int b = 0; b < GT / 32; ++b) acc[a][b] = 0.0f;
#pragma unroll 4
            for (int q = 0; q < 32; ++q) {
                float li[GT / 16], lc[GT / 32];
#pragma unroll
                for (int a = 0; a < GT / 16; ++a) li[a] = L[(ty + 16 * a) * DB_LD + o + q];
#pragma unroll
                for (int b = 0; b < GT / 32; ++b) lc[b] = L[(tx + 32 * b) * DB_LD + o + q];
#pragma unroll
                for (int a = 0; a < GT / 16; ++a)
#pragma unroll
                    for (int b = 0; b < GT / 32; ++b) acc[a][b] += li[a] * lc[b];
            }
#pragma unroll
            for (int a = 0; a < GT / 16; ++a) {
                const int i = ty + 16 * a;
#pragma unroll
                for (int b = 0; b < GT / 32; ++b) {
                    const int c = tx + 32 * b;
                    if (i >= R0 && c >= R0 && c <= i) L[i * DB_LD + c] -= acc[a][b];
                }
            }
            __syncthreads();
        }
    }
    // X = L^-1 by block rows: T = sum_j L_ij X_j. (columns < 32 i), X_i. = -W_i T
    for (int ib = 1; ib < 4; ++ib) {
        const int o = ib * 32, nc = ib * 32;
        for (int e = t; e < 32 * nc; e += DB_THREADS) {
            const int q = e / nc, col = e % nc;
            float acc = 0.0f;
            for (int m = (col >> 5) << 5; m < o; ++m) acc += L[(o + q) * DB_LD + m] * X[m * DB_LD + col];
            T[q * 97 + col] = acc;
        }
        __syncthreads();
        for (int e = t; e < 32 * nc; e += DB_THREADS) {
            const int q = e / nc, col = e % nc;
            float acc = 0.0f;
            for (int p = 0; p <= q; ++p) acc += W[(ib * 32 + q) * 33 + p] * T[p * 97 + col];
            X[(o + q) * DB_LD + col] = -acc;
        }
        __syncthreads();
    }
    for (int e = t; e < GT * GT; e += DB_THREADS) {
        const int r = e >> 7, c = e & (GT - 1);
        Akk[(long long)r * ld + c] = c <= r ? L[r * DB_LD + c] : 0.0f;
        Dinv[r * GT + c] = c <= r ? X[r * DB_LD + c] : 0.0f;
    }
}

// XT block (i, i) = Dinv_i^T
__global__ void k_put_diag_t(float* __restrict__ XT, int ld, int i, const float* __restrict__ Dinv) {
    const int t = threadIdx.x;
    for (int r = 0; r < GT; ++r) XT[(long long)(i * GT + r) * ld + i * GT + t] = Dinv[t * GT + r];
}

// X block (i, i) = Dinv_i (lower, zeros above)
__global__ void k_put_diag(float* __restrict__ X, int ld, int i, const float* __restrict__ Dinv) {
    const int t = threadIdx.x;
    for (int r = 0; r < GT; ++r) X[(long long)(i * GT + r) * ld + i * GT + t] = Dinv[r * GT + t];
}

// dst[c][r] = src[r][c] for a rows x cols block (both multiples of 32),
// through 32 x 33 shared-memory tiles; blocks of 32 x 8 threads
__global__ void k_transpose_block(const float* __restrict__ src, int lds, float* __restrict__ dst, int ldd, int rows,
                                  int cols) {
    __shared__ float tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    if (r0 >= rows || c0 >= cols) return;
    for (int y = threadIdx.y; y < 32; y += 8)
        tile[y][threadIdx.x] = src[(long long)(r0 + y) * lds + c0 + threadIdx.x];
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += 8)
        dst[(long long)(c0 + y) * ldd + r0 + threadIdx.x] = tile[threadIdx.x][y];
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

// shared-memory limits, raised once per device (function attributes belong to
// the device that is current when they are set)
void set_attributes() {
    static PerDeviceOnce once;
    once.run([] {
        IBR_CUDA_TRY(cudaFuncSetAttribute(k_gemm_tf32x3, cudaFuncAttributeMaxDynamicSharedMemorySize, GEMM_SMEM));
        IBR_CUDA_TRY(cudaFuncSetAttribute(k_diag_block, cudaFuncAttributeMaxDynamicSharedMemorySize, DB_SMEM));
    });
}

}  // namespace

void gemm_tf32x3(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc, float alpha,
                 float beta, bool lower_only, int* err_dev, cudaStream_t s) {
    if (M % GT || N % GT || K % GK || K == 0 || lda % 4 || ldb % 4)
        throw Error{IBR_EINVAL, "gemm_tf32x3: M, N must be multiples of 128, K a positive multiple of 32, lda and ldb "
                                "multiples of 4"};
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15)
        throw Error{IBR_EINVAL, "gemm_tf32x3: A and B must be 16-byte aligned"};
    if (M == 0 || N == 0) return;
    set_attributes();
    // pack A (and B unless it is the same matrix) into TF32 hi / lo slices
    const bool same = A == B && lda == ldb && M == N;
    const size_t ea = (size_t)M * K, eb = same ? 0 : (size_t)N * K;
    float* pk = nullptr;
    IBR_CUDA_TRY(cudaMallocAsync(&pk, (2 * ea + 2 * eb) * sizeof(float), s));
    float *pah = pk, *pal = pk + ea, *pbh = same ? pah : pk + 2 * ea, *pbl = same ? pal : pk + 2 * ea + eb;
    {
        ProfScope ps(KID_TC_GEMM, s, 12.0 * (double)(ea + eb));
        k_pack_tf32<<<grid_1d((long long)ea / 4, 256), 256, 0, s>>>(A, lda, M, K, pah, pal);
        IBR_CHECK_LAUNCH();
        if (!same) {
            k_pack_tf32<<<grid_1d((long long)eb / 4, 256), 256, 0, s>>>(B, ldb, N, K, pbh, pbl);
            IBR_CHECK_LAUNCH();
        }
    }
    {
        // executed tensor FLOPs: three TF32 products per output over the tiles computed
        const double tiles = lower_only ? (double)(M / GT) * (M / GT + 1) / 2.0 : (double)(M / GT) * (N / GT);
        ProfScope ps(KID_TC_GEMM, s, 8.0 * ((double)M * K + (double)N * K) + 4.0 * 2.0 * M * N,
                     3.0 * 2.0 * tiles * GT * GT * (double)K);
        dim3 grid(N / GT, M / GT);
        k_gemm_tf32x3<<<grid, GT, GEMM_SMEM, s>>>(K, pah, pal, pbh, pbl, C, ldc, alpha, beta, lower_only ? 1 : 0,
                                                  err_dev);
        IBR_CHECK_LAUNCH();
    }
    IBR_CUDA_TRY(cudaFreeAsync(pk, s));
}

// X[b0:b1, b0:b1] = L[b0:b1, b0:b1]^-1 (blocks of 128; X lower, XT = X^T
// upper, both row-major np x np, their diagonal blocks already set) by
// splitting at m: X11 and X22 recursively, then
//   TT  = XT11 L21^T        ( = (L21 X11)^T, s1 x s2 )
//   X21 = -X22 TT^T         ( = -X22 L21 X11, s2 x s1 ), XT12 = X21^T.
// The zero upper part of X22 and lower part of XT11 enter the products as is.
void trtri_rec(int b0, int b1, int np, const float* L, float* X, float* XT, float* TT, int* err_dev, cudaStream_t s) {
    if (b1 - b0 <= 1) return;
    const int m = b0 + (b1 - b0) / 2;
    trtri_rec(b0, m, np, L, X, XT, TT, err_dev, s);
    trtri_rec(m, b1, np, L, X, XT, TT, err_dev, s);
    const int s1 = (m - b0) * GT, s2 = (b1 - m) * GT;
    const long long o11 = (long long)b0 * GT * np + (long long)b0 * GT;
    const long long o21 = (long long)m * GT * np + (long long)b0 * GT;
    const long long o22 = (long long)m * GT * np + (long long)m * GT;
    const long long o12 = (long long)b0 * GT * np + (long long)m * GT;
    gemm_tf32x3(s1, s2, s1, XT + o11, np, L + o21, np, TT, s2, 1.f, 0.f, false, err_dev, s);
    gemm_tf32x3(s2, s1, s2, X + o22, np, TT, s2, X + o21, np, -1.f, 0.f, false, err_dev, s);
    ProfScope ps(KID_SPD_INV, s, 8.0 * s1 * s2);
    dim3 grid(s1 / 32, s2 / 32), blk(32, 8);
    k_transpose_block<<<grid, blk, 0, s>>>(X + o21, np, XT + o12, np, s2, s1);
    IBR_CHECK_LAUNCH();
}

// M (n x n SPD, FP32, row-major) -> M^-1 on the tensor cores: padded to a
// multiple of 128 with an identity block, blocked right-looking Cholesky
// (diagonal blocks on CUDA cores, panel A_ik L_kk^-T and trailing update
// A_ij -= L_ik L_jk^T as tensor-core products), X = L^-1 and X^T
// recursively by 2 x 2 blocks (trtri_rec), then M^-1 = X^T (X^T)^T (lower
// tiles) and the symmetric n x n corner.
void spd_inverse_tc(int n, float* M, int* info_dev, double min_pivot, double pad, int* err_dev, cudaStream_t s) {
    set_attributes();
    const int np = (n + GT - 1) / GT * GT;
    const int nb = np / GT;
    float *P = nullptr, *X = nullptr, *XT = nullptr, *TT = nullptr, *Dinv = nullptr;
    IBR_CUDA_TRY(cudaMallocAsync(&P, (size_t)np * np * sizeof(float), s));
    IBR_CUDA_TRY(cudaMallocAsync(&X, (size_t)np * np * sizeof(float), s));
    IBR_CUDA_TRY(cudaMallocAsync(&XT, (size_t)np * np * sizeof(float), s));
    // the largest s1 x s2 product of the recursion: s1 + s2 <= np, so s1 s2 <= np^2 / 4
    IBR_CUDA_TRY(cudaMallocAsync(&TT, ((size_t)np * np / 4 + (size_t)GT * GT) * sizeof(float), s));
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
            k_diag_block<<<1, DB_THREADS, DB_SMEM, s>>>(
                P, np, k, Dinv + (long long)k * GT * GT, info_dev, (float)min_pivot);
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
    // X = L^-1 (and X^T) by the recursive 2 x 2 block formula
    // X21 = -X22 L21 X11: every level's products span the whole block
    IBR_CUDA_TRY(cudaMemsetAsync(X, 0, (size_t)np2 * sizeof(float), s));
    IBR_CUDA_TRY(cudaMemsetAsync(XT, 0, (size_t)np2 * sizeof(float), s));
    for (int i = 0; i < nb; ++i) {
        ProfScope ps(KID_SPD_INV, s, 4.0 * 3 * GT * GT);
        k_put_diag<<<1, GT, 0, s>>>(X, np, i, Dinv + (long long)i * GT * GT);
        IBR_CHECK_LAUNCH();
        k_put_diag_t<<<1, GT, 0, s>>>(XT, np, i, Dinv + (long long)i * GT * GT);
        IBR_CHECK_LAUNCH();
    }
    trtri_rec(0, nb, np, P, X, XT, TT, err_dev, s);
    gemm_tf32x3(np, np, np, XT, np, XT, np, P, np, 1.f, 0.f, true, err_dev, s);
    {
        ProfScope ps(KID_SPD_INV, s, 4.0 * 2.0 * n * n);
        k_sym_out<<<grid_1d((long long)n * n, 256), 256, 0, s>>>(n, np, P, M);
        IBR_CHECK_LAUNCH();
    }
    IBR_CUDA_TRY(cudaFreeAsync(P, s));
    IBR_CUDA_TRY(cudaFreeAsync(X, s));
    IBR_CUDA_TRY(cudaFreeAsync(XT, s));
    IBR_CUDA_TRY(cudaFreeAsync(TT, s));
    IBR_CUDA_TRY(cudaFreeAsync(Dinv, s));
}

}  // namespace ibr
