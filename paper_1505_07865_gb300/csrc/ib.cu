// Fluid-marker coupling (Sec. III.A) and rigid-body kinematics (Sec. II).
//
//  (J v)_i^a = sum_k v_k^a prod_b phi((q_i - r_k^a)_b / h)
//  (S L)_k^a = h^-d sum_i L_i^a prod_b phi((q_i - r_k^a)_b / h)
//
// with the 4-point Peskin kernel or the six-point kernel of Bao, Kaye and
// Peskin as phi (window of g.kw = 4 or 6 nodes per axis).  Spreading is a
// face-major gather: the
// (face, marker, weight) triples of S are sorted by face once per geometry,
// so each touched face is summed by one thread in a fixed order (no atomics,
// bitwise reproducible).
#include "ibr_internal.cuh"

namespace ibr {
namespace {

__global__ void k_positions(int d, int N, const double* __restrict__ rb, const int* __restrict__ body,
                            const double* __restrict__ xcR, double L0, double L1, double L2, double* __restrict__ q,
                            double* __restrict__ rel) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double* P = xcR + 12 * body[i];  // x_c[3], R[9] row-major
    double r[3] = {rb[i * d + 0], rb[i * d + 1], d == 3 ? rb[i * d + 2] : 0.0};
    const double Ls[3] = {L0, L1, L2};
    for (int a = 0; a < d; ++a) {
        double v = P[3 + 3 * a + 0] * r[0] + P[3 + 3 * a + 1] * r[1] + P[3 + 3 * a + 2] * r[2];
        rel[i * d + a] = v;
        double x = P[a] + v;
        if (Ls[a] > 0.0) {
            x -= Ls[a] * floor(x / Ls[a]);
            if (x >= Ls[a]) x -= Ls[a];
        }
        q[i * d + a] = x;
    }
}

// For component a, axis b and window node m (t = (i*d + a)*d + b):
// idx[t*kw + m] = the stored node the window node maps to and w[t*kw + m] its
// signed weight.  Periodic axes wrap.  On a wall axis the field is extended
// beyond the walls by its mirror image with a sign (App. D): the component
// tangential to the wall (cell-centred along b) by ghost = -mirror, the
// normal component (faces 0..n on b, face 0 and face n on the walls) by
// u(-k) = -u(k), u(n+k) = -u(n-k), and the wall faces themselves carry
// boundary data, not unknowns: weight 0.
__global__ void k_weights(Geo g, int N, const double* __restrict__ q, int* __restrict__ idx, double* __restrict__ w64,
                          float* __restrict__ w32) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int d = g.d;
    if (t >= N * d * d) return;
    int i = t / (d * d);
    int a = (t / d) % d;
    int b = t % d;
    double off = (a == b) ? 0.0 : 0.5;
    double s = q[i * d + b] / g.h - off;
    const int kw = g.kw;
    int j0 = 0;
    double wts[6];
    kernel_window(kw, s, j0, wts);
    int nb = b == 0 ? g.n0 : (b == 1 ? g.n1 : g.n2);
    bool wall = (g.wall >> b) & 1;
    for (int m = 0; m < kw; ++m) {
        double ww = wts[m];
        int j = j0 + m;
        int st;
        if (!wall) {
            st = j % nb;
            if (st < 0) st += nb;
        } else if (a == b) {
            if (j == 0 || j == nb) {
                st = 0;
                ww = 0.0;
            } else if (j < 0) {
                st = -j;
                ww = -ww;
            } else if (j > nb) {
                st = 2 * nb - j;
                ww = -ww;
            } else {
                st = j;
            }
        } else {
            if (j < 0) {
                st = -j - 1;
                ww = -ww;
            } else if (j >= nb) {
                st = 2 * nb - 1 - j;
                ww = -ww;
            } else {
                st = j;
            }
        }
        idx[t * kw + m] = st;
        w64[t * kw + m] = ww;
        w32[t * kw + m] = (float)ww;
    }
}

// entry e of the (marker component, window cell) list: kw^D window cells per
// marker component, window node m_b = (c / kw^b) mod kw on axis b
template <int D>
__device__ __forceinline__ void entry_face(const Geo& g, const int* __restrict__ idx, const double* __restrict__ w64,
                                           long long e, long long& key, double& wt, int& mcomp) {
    const int kw = g.kw;
    const int S = D == 3 ? kw * kw * kw : kw * kw;
    int c = (int)(e % S);
    long long ia = e / S;  // i*D + a
    int a = (int)(ia % D);
    mcomp = (int)ia;
    const int ns[3] = {g.n0, g.n1, g.n2};
    long long cell = 0, stride = 1;
    wt = 1.0;
#pragma unroll
    for (int b = 0; b < D; ++b) {
        int m = c % kw;
        c /= kw;
        long long t = ia * D + b;
        int j = idx[t * kw + m];
        cell += j * stride;
        stride *= ns[b];
        wt *= w64[t * kw + m];
    }
    key = (long long)a * g.ncell + cell;
}

template <int D>
__global__ void k_keys(Geo g, long long E, long long P, const int* __restrict__ idx, const double* __restrict__ w64,
                       unsigned long long* __restrict__ keys) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= P) return;
    if (e >= E) {
        keys[e] = ~0ULL;
        return;
    }
    long long key;
    double wt;
    int mc;
    entry_face<D>(g, idx, w64, e, key, wt, mc);
    keys[e] = ((unsigned long long)key << 32) | (unsigned long long)e;
}

// ---- bitonic sort of P = 2^p keys (ascending) ------------------------------
constexpr int BS_ELEMS = 2048;

__device__ __forceinline__ void cmp_swap(unsigned long long& x, unsigned long long& y, bool asc) {
    if ((x > y) == asc) {
        unsigned long long t = x;
        x = y;
        y = t;
    }
}

// all stages with size <= 2048 inside one CTA's chunk
__global__ void __launch_bounds__(1024) k_bitonic_local(unsigned long long* keys) {
    __shared__ unsigned long long s[BS_ELEMS];
    long long base = (long long)blockIdx.x * BS_ELEMS;
    int t = threadIdx.x;
    s[t] = keys[base + t];
    s[t + 1024] = keys[base + t + 1024];
    __syncthreads();
    for (int size = 2; size <= BS_ELEMS; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            int pos = 2 * t - (t & (stride - 1));
            bool asc = (((base + pos) & size) == 0);
            cmp_swap(s[pos], s[pos + stride], asc);
            __syncthreads();
        }
    }
    keys[base + t] = s[t];
    keys[base + t + 1024] = s[t + 1024];
}

// one global compare-exchange pass (stride >= 2048)
__global__ void k_bitonic_global(unsigned long long* keys, long long P, long long size, long long stride) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= P / 2) return;
    long long pos = 2 * t - (t & (stride - 1));
    bool asc = ((pos & size) == 0);
    unsigned long long x = keys[pos], y = keys[pos + stride];
    if ((x > y) == asc) {
        keys[pos] = y;
        keys[pos + stride] = x;
    }
}

// strides 1024..1 of a stage of the given size, inside one CTA
__global__ void __launch_bounds__(1024) k_bitonic_merge_local(unsigned long long* keys, long long size) {
    __shared__ unsigned long long s[BS_ELEMS];
    long long base = (long long)blockIdx.x * BS_ELEMS;
    int t = threadIdx.x;
    s[t] = keys[base + t];
    s[t + 1024] = keys[base + t + 1024];
    __syncthreads();
    for (int stride = BS_ELEMS >> 1; stride > 0; stride >>= 1) {
        int pos = 2 * t - (t & (stride - 1));
        bool asc = (((base + pos) & size) == 0);
        cmp_swap(s[pos], s[pos + stride], asc);
        __syncthreads();
    }
    keys[base + t] = s[t];
    keys[base + t + 1024] = s[t + 1024];
}

// segment heads: flag[t] = 1 if key(t) differs from key(t-1)
__global__ void k_seg_flags(long long E, const unsigned long long* __restrict__ keys, int* __restrict__ flag) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= E) return;
    flag[t] = (t == 0 || (keys[t] >> 32) != (keys[t - 1] >> 32)) ? 1 : 0;
}

// exclusive scan of flag[0..E) into pos[0..E], single CTA (set-up only)
__global__ void __launch_bounds__(1024) k_scan_single(long long E, const int* __restrict__ flag, int* __restrict__ pos) {
    __shared__ int sm[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long c0 = 0; c0 < E; c0 += 1024) {
        long long t = c0 + threadIdx.x;
        int v = t < E ? flag[t] : 0;
        sm[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            int add = threadIdx.x >= o ? sm[threadIdx.x - o] : 0;
            __syncthreads();
            sm[threadIdx.x] += add;
            __syncthreads();
        }
        if (t < E) pos[t] = carry + sm[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += sm[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) pos[E] = carry;
}

template <int D>
__global__ void k_seg_build(Geo g, long long E, const unsigned long long* __restrict__ keys,
                            const int* __restrict__ flag, const int* __restrict__ pos, const int* __restrict__ idx,
                            const double* __restrict__ w64, long long* __restrict__ face, int* __restrict__ off,
                            int* __restrict__ ent_m, double* __restrict__ ew64, float* __restrict__ ew32) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= E) return;
    long long e = (long long)(keys[t] & 0xffffffffULL);
    long long key;
    double wt;
    int mc;
    entry_face<D>(g, idx, w64, e, key, wt, mc);
    ent_m[t] = mc;
    ew64[t] = wt;
    ew32[t] = (float)wt;
    if (flag[t]) {
        int sidx = pos[t];
        face[sidx] = key;
        off[sidx] = (int)t;
    }
}

__global__ void k_set_int(int* p, int v) { *p = v; }

template <typename T>
__global__ void k_spread_gather(long long F, const long long* __restrict__ face, const int* __restrict__ off,
                                const int* __restrict__ ent_m, const T* __restrict__ ew, const T* __restrict__ lam,
                                T* __restrict__ y, T scale) {
    long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (f >= F) return;
    T s = T(0);
    int e1 = off[f + 1];
    for (int e = off[f]; e < e1; ++e) s += ew[e] * lam[ent_m[e]];
    y[face[f]] += scale * s;
}

// one warp per marker; lanes stride the KW^D support of each component
template <int D, int KW, typename T, typename Tadd>
__global__ void k_interp(Geo g, int N, const int* __restrict__ idx, const T* __restrict__ w, const T* __restrict__ v,
                         T* __restrict__ out, T sign, const Tadd* __restrict__ add, T add_scale) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= N) return;
    const int S = D == 3 ? KW * KW * KW : KW * KW;
    const int ns[3] = {g.n0, g.n1, g.n2};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const T* va = v + a * g.ncell;
        long long ia = (long long)warp * D + a;
        T acc = T(0);
        for (int c = lane; c < S; c += 32) {
            long long cell = 0, stride = 1;
            T wt = T(1);
            int cc = c;
#pragma unroll
            for (int b = 0; b < D; ++b) {
                const int m = cc % KW;
                cc /= KW;
                long long t = ia * D + b;
                int j = idx[t * KW + m];
                cell += j * stride;
                stride *= ns[b];
                wt *= w[t * KW + m];
            }
            acc += wt * va[cell];
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            T r = sign * acc;
            if (add) r += add_scale * (T)add[ia];
            out[ia] = r;
        }
    }
}

template <typename T>
__global__ void k_lam_sum(int d, int N, const T* __restrict__ lam, double scale, double* __restrict__ shift) {
    __shared__ double sm[3][32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int a = 0; a < d; ++a) {
        double s = 0.0;
        for (int i = threadIdx.x; i < N; i += blockDim.x) s += (double)lam[(long long)i * d + a];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) sm[a][wid] = s;
    }
    __syncthreads();
    if (wid == 0) {
        for (int a = 0; a < d; ++a) {
            double s = lane < (int)(blockDim.x >> 5) ? sm[a][lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) shift[a] = scale * s;
        }
    }
}

__global__ void k_rigid_K(int d, int N, const double* __restrict__ rel, const int* __restrict__ body,
                          const double* __restrict__ UO, double* __restrict__ V, double sign) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int nr = d == 2 ? 1 : 3;
    const double* u = UO + (long long)body[i] * (d + nr);
    const double* r = rel + (long long)i * d;
    if (d == 2) {
        double w = u[2];
        V[i * 2 + 0] = sign * (u[0] - w * r[1]);
        V[i * 2 + 1] = sign * (u[1] + w * r[0]);
    } else {
        const double* O = u + 3;
        V[i * 3 + 0] = sign * (u[0] + O[1] * r[2] - O[2] * r[1]);
        V[i * 3 + 1] = sign * (u[1] + O[2] * r[0] - O[0] * r[2]);
        V[i * 3 + 2] = sign * (u[2] + O[0] * r[1] - O[1] * r[0]);
    }
}

// one CTA per body: [sum lam ; sum rel x lam]
__global__ void k_rigid_KT(int d, const int* __restrict__ bstart, const double* __restrict__ rel,
                           const double* __restrict__ lam, double* __restrict__ FT) {
    int b = blockIdx.x;
    int i0 = bstart[b], i1 = bstart[b + 1];
    int nr = d == 2 ? 1 : 3;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const double* r = rel + (long long)i * d;
        const double* l = lam + (long long)i * d;
        if (d == 2) {
            acc[0] += l[0];
            acc[1] += l[1];
            acc[2] += r[0] * l[1] - r[1] * l[0];
        } else {
            acc[0] += l[0];
            acc[1] += l[1];
            acc[2] += l[2];
            acc[3] += r[1] * l[2] - r[2] * l[1];
            acc[4] += r[2] * l[0] - r[0] * l[2];
            acc[5] += r[0] * l[1] - r[1] * l[0];
        }
    }
    __shared__ double sm[6][32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int q = 0; q < d + nr; ++q) {
        double s = acc[q];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) sm[q][wid] = s;
    }
    __syncthreads();
    if (wid == 0) {
        for (int q = 0; q < d + nr; ++q) {
            double s = lane < (int)(blockDim.x >> 5) ? sm[q][lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) FT[(long long)b * (d + nr) + q] = s;
        }
    }
}

}  // namespace

void markers_positions(int d, int N, const double* rbody, const int* body, const double* xc_R, const double* Lbox,
                       double* q, double* rel, cudaStream_t s) {
    ProfScope ps(KID_MARKERS, s, 0.0);
    k_positions<<<grid_1d(N, 128), 128, 0, s>>>(d, N, rbody, body, xc_R, Lbox[0], Lbox[1], d == 3 ? Lbox[2] : 0.0, q,
                                                  rel);
    IBR_CHECK_LAUNCH();
}

void markers_weights(const Geo& g, int N, const double* q, int* idx, double* w64, float* w32, cudaStream_t s) {
    int n = N * g.d * g.d;
    ProfScope ps(KID_MARKERS, s, 0.0);
    k_weights<<<grid_1d(n, 128), 128, 0, s>>>(g, N, q, idx, w64, w32);
    IBR_CHECK_LAUNCH();
}

void markers_build_gather(const Geo& g, MarkerData& md, cudaStream_t s) {
    const int S = g.d == 3 ? g.kw * g.kw * g.kw : g.kw * g.kw;
    long long E = (long long)md.N * g.d * S;
    long long P = BS_ELEMS;
    while (P < E) P <<= 1;
    ProfScope ps(KID_MARKERS, s, 0.0);
    unsigned long long* keys = nullptr;
    int* flag = nullptr;
    int* pos = nullptr;
    IBR_CUDA_TRY(cudaMallocAsync(&keys, P * sizeof(unsigned long long), s));
    IBR_CUDA_TRY(cudaMallocAsync(&flag, E * sizeof(int), s));
    IBR_CUDA_TRY(cudaMallocAsync(&pos, (E + 1) * sizeof(int), s));
    if (g.d == 3)
        k_keys<3><<<grid_1d(P, 256), 256, 0, s>>>(g, E, P, md.idx, md.w64, keys);
    else
        k_keys<2><<<grid_1d(P, 256), 256, 0, s>>>(g, E, P, md.idx, md.w64, keys);
    IBR_CHECK_LAUNCH();
    int nchunks = (int)(P / BS_ELEMS);
    k_bitonic_local<<<nchunks, 1024, 0, s>>>(keys);
    IBR_CHECK_LAUNCH();
    for (long long size = 2 * BS_ELEMS; size <= P; size <<= 1) {
        for (long long stride = size >> 1; stride >= BS_ELEMS; stride >>= 1) {
            k_bitonic_global<<<grid_1d(P / 2, 256), 256, 0, s>>>(keys, P, size, stride);
            IBR_CHECK_LAUNCH();
        }
        k_bitonic_merge_local<<<nchunks, 1024, 0, s>>>(keys, size);
        IBR_CHECK_LAUNCH();
    }
    k_seg_flags<<<grid_1d(E, 256), 256, 0, s>>>(E, keys, flag);
    IBR_CHECK_LAUNCH();
    k_scan_single<<<1, 1024, 0, s>>>(E, flag, pos);
    IBR_CHECK_LAUNCH();
    int F = 0;
    IBR_CUDA_TRY(cudaMemcpyAsync(&F, pos + E, sizeof(int), cudaMemcpyDeviceToHost, s));
    IBR_CUDA_TRY(cudaStreamSynchronize(s));
    md.E = E;
    md.F = F;
    IBR_CUDA_TRY(cudaMalloc(&md.face, (size_t)F * sizeof(long long)));
    IBR_CUDA_TRY(cudaMalloc(&md.off, (size_t)(F + 1) * sizeof(int)));
    IBR_CUDA_TRY(cudaMalloc(&md.ent_m, (size_t)E * sizeof(int)));
    IBR_CUDA_TRY(cudaMalloc(&md.ent_w64, (size_t)E * sizeof(double)));
    IBR_CUDA_TRY(cudaMalloc(&md.ent_w32, (size_t)E * sizeof(float)));
    if (g.d == 3)
        k_seg_build<3><<<grid_1d(E, 256), 256, 0, s>>>(g, E, keys, flag, pos, md.idx, md.w64, md.face, md.off,
                                                      md.ent_m, md.ent_w64, md.ent_w32);
    else
        k_seg_build<2><<<grid_1d(E, 256), 256, 0, s>>>(g, E, keys, flag, pos, md.idx, md.w64, md.face, md.off,
                                                      md.ent_m, md.ent_w64, md.ent_w32);
    IBR_CHECK_LAUNCH();
    k_set_int<<<1, 1, 0, s>>>(md.off + F, (int)E);
    IBR_CHECK_LAUNCH();
    IBR_CUDA_TRY(cudaFreeAsync(keys, s));
    IBR_CUDA_TRY(cudaFreeAsync(flag, s));
    IBR_CUDA_TRY(cudaFreeAsync(pos, s));
}

template <typename T>
void spread_gather(const MarkerData& md, const T* lam, T* y, double scale, cudaStream_t s) {
    if (md.F == 0) return;
    const T* ew = nullptr;
    if (sizeof(T) == 8)
        ew = reinterpret_cast<const T*>(md.ent_w64);
    else
        ew = reinterpret_cast<const T*>(md.ent_w32);
    ProfScope ps(KID_SPREAD, s, (double)md.F * (8 + 4 + 2 * sizeof(T)) + (double)md.E * (4 + 2 * sizeof(T)));
    k_spread_gather<T><<<grid_1d(md.F, 128), 128, 0, s>>>(md.F, md.face, md.off, md.ent_m, ew, lam, y, (T)scale);
    IBR_CHECK_LAUNCH();
}

template <typename T, typename Tadd>
void interp(const Geo& g, const MarkerData& md, const T* v, T* out, double sign, const Tadd* add, cudaStream_t s,
            double add_scale) {
    const T* w = sizeof(T) == 8 ? reinterpret_cast<const T*>(md.w64) : reinterpret_cast<const T*>(md.w32);
    int threads = 128;
    int blocks = grid_1d((long long)md.N * 32, threads);
    const int kw = g.kw;
    ProfScope ps(KID_INTERP, s,
                 (double)md.N * g.d * ((g.d == 3 ? kw * kw * kw : kw * kw) * sizeof(T) + g.d * kw * sizeof(T) + sizeof(T)));
    if (g.d == 3) {
        if (kw == 6)
            k_interp<3, 6, T, Tadd><<<blocks, threads, 0, s>>>(g, md.N, md.idx, w, v, out, (T)sign, add, (T)add_scale);
        else
            k_interp<3, 4, T, Tadd><<<blocks, threads, 0, s>>>(g, md.N, md.idx, w, v, out, (T)sign, add, (T)add_scale);
    } else {
        if (kw == 6)
            k_interp<2, 6, T, Tadd><<<blocks, threads, 0, s>>>(g, md.N, md.idx, w, v, out, (T)sign, add, (T)add_scale);
        else
            k_interp<2, 4, T, Tadd><<<blocks, threads, 0, s>>>(g, md.N, md.idx, w, v, out, (T)sign, add, (T)add_scale);
    }
    IBR_CHECK_LAUNCH();
}

template <typename T>
void lam_sum(int d, int N, const T* lam, double scale, double* shift, cudaStream_t s) {
    ProfScope ps(KID_LAMSUM, s, (double)N * d * sizeof(T));
    k_lam_sum<T><<<1, 256, 0, s>>>(d, N, lam, scale, shift);
    IBR_CHECK_LAUNCH();
}

void rigid_K(int d, int N, const double* rel, const int* body, const double* UO, double* V, double sign,
             cudaStream_t s) {
    ProfScope ps(KID_RIGID_K, s, (double)N * d * 8 * 3);
    k_rigid_K<<<grid_1d(N, 128), 128, 0, s>>>(d, N, rel, body, UO, V, sign);
    IBR_CHECK_LAUNCH();
}

void rigid_KT(int d, int B, const int* body_start, const double* rel, const double* lam, double* FT, cudaStream_t s) {
    ProfScope ps(KID_RIGID_KT, s, 0.0);
    k_rigid_KT<<<B, 256, 0, s>>>(d, body_start, rel, lam, FT);
    IBR_CHECK_LAUNCH();
}

template void spread_gather<double>(const MarkerData&, const double*, double*, double, cudaStream_t);
template void spread_gather<float>(const MarkerData&, const float*, float*, double, cudaStream_t);
template void interp<double, double>(const Geo&, const MarkerData&, const double*, double*, double, const double*,
                                     cudaStream_t, double);
template void interp<float, double>(const Geo&, const MarkerData&, const float*, float*, double, const double*,
                                    cudaStream_t, double);
template void lam_sum<double>(int, int, const double*, double, double*, cudaStream_t);
template void lam_sum<float>(int, int, const float*, double, double*, cudaStream_t);

}  // namespace ibr

// ---- free kinematics (bodies with unknown rigid velocity) ------------------
namespace ibr {
namespace {

// out[i] += sign * (K U_f)_i on the markers of free bodies (bfree[b] = free
// index or -1); U_f body-major, nr = d + rot entries per free body
__global__ void k_rigid_K_free(int d, int N, const double* __restrict__ rel, const int* __restrict__ body,
                               const int* __restrict__ bfree, const double* __restrict__ Uf, double* __restrict__ out,
                               double sign) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int fb = bfree[body[i]];
    if (fb < 0) return;
    int nr = d == 2 ? 3 : 6;
    const double* u = Uf + (long long)fb * nr;
    const double* r = rel + (long long)i * d;
    if (d == 2) {
        out[i * 2 + 0] += sign * (u[0] - u[2] * r[1]);
        out[i * 2 + 1] += sign * (u[1] + u[2] * r[0]);
    } else {
        const double* O = u + 3;
        out[i * 3 + 0] += sign * (u[0] + O[1] * r[2] - O[2] * r[1]);
        out[i * 3 + 1] += sign * (u[1] + O[2] * r[0] - O[0] * r[2]);
        out[i * 3 + 2] += sign * (u[2] + O[0] * r[1] - O[1] * r[0]);
    }
}

// one CTA per body: [sum lam; sum rel x lam] of a free body written at
// out[fb*nr .. ) (bodies with bfree[b] < 0 are skipped)
template <typename Tl>
__global__ void k_rigid_KT_free(int d, const int* __restrict__ bstart, const int* __restrict__ bfree,
                                const double* __restrict__ rel, const Tl* __restrict__ lam, double* __restrict__ out) {
    int b = blockIdx.x;
    int fb = bfree[b];
    if (fb < 0) return;
    int i0 = bstart[b], i1 = bstart[b + 1];
    int nr = d == 2 ? 3 : 6;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const double* r = rel + (long long)i * d;
        double l0 = (double)lam[(long long)i * d], l1 = (double)lam[(long long)i * d + 1];
        if (d == 2) {
            acc[0] += l0;
            acc[1] += l1;
            acc[2] += r[0] * l1 - r[1] * l0;
        } else {
            double l2 = (double)lam[(long long)i * d + 2];
            acc[0] += l0;
            acc[1] += l1;
            acc[2] += l2;
            acc[3] += r[1] * l2 - r[2] * l1;
            acc[4] += r[2] * l0 - r[0] * l2;
            acc[5] += r[0] * l1 - r[1] * l0;
        }
    }
    __shared__ double sm[6][32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int q = 0; q < nr; ++q) {
        double s = acc[q];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) sm[q][wid] = s;
    }
    __syncthreads();
    if (wid == 0) {
        for (int q = 0; q < nr; ++q) {
            double s = lane < (int)(blockDim.x >> 5) ? sm[q][lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) out[(long long)fb * nr + q] = s;
        }
    }
}

// lam[e] += sum_c X[c*dN + e] * U_f[fb(e)*nr + c] on free bodies' markers
template <typename T>
__global__ void k_lam_add_XU(int d, int N, const int* __restrict__ body, const int* __restrict__ bfree,
                             const T* __restrict__ X, const double* __restrict__ Uf, T* __restrict__ lam) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long dN = (long long)N * d;
    if (e >= dN) return;
    int fb = bfree[body[e / d]];
    if (fb < 0) return;
    int nr = d == 2 ? 3 : 6;
    double s = 0.0;
    for (int c = 0; c < nr; ++c) s += (double)X[c * dN + e] * Uf[(long long)fb * nr + c];
    lam[e] = (T)((double)lam[e] + s);
}

// per free body (one thread each): U = Nb (r - s), Nb nr x nr row-major
__global__ void k_body_solve(int nfree, int nr, const double* __restrict__ Nb, const double* __restrict__ r,
                             const double* __restrict__ s, double* __restrict__ U) {
    int fb = blockIdx.x * blockDim.x + threadIdx.x;
    if (fb >= nfree) return;
    const double* A = Nb + (long long)fb * nr * nr;
    for (int a = 0; a < nr; ++a) {
        double acc = 0.0;
        for (int c = 0; c < nr; ++c) acc += A[a * nr + c] * (r[fb * nr + c] - s[fb * nr + c]);
        U[fb * nr + a] = acc;
    }
}

// in-place inverse of each free body's nr x nr block (Gauss-Jordan with
// partial pivoting, FP64, one thread per body); info set if singular
__global__ void k_small_inverse(int nfree, int nr, double* __restrict__ A, int* __restrict__ info) {
    int fb = blockIdx.x * blockDim.x + threadIdx.x;
    if (fb >= nfree) return;
    double* M = A + (long long)fb * nr * nr;
    double a[6][12];
    for (int i = 0; i < nr; ++i)
        for (int j = 0; j < 2 * nr; ++j) a[i][j] = j < nr ? M[i * nr + j] : (j - nr == i ? 1.0 : 0.0);
    for (int c = 0; c < nr; ++c) {
        int p = c;
        for (int i = c + 1; i < nr; ++i)
            if (fabs(a[i][c]) > fabs(a[p][c])) p = i;
        if (!(fabs(a[p][c]) > 0.0)) {
            atomicExch(info, 1);
            return;
        }
        if (p != c)
            for (int j = 0; j < 2 * nr; ++j) {
                double t = a[c][j];
                a[c][j] = a[p][j];
                a[p][j] = t;
            }
        double iv = 1.0 / a[c][c];
        for (int j = 0; j < 2 * nr; ++j) a[c][j] *= iv;
        for (int i = 0; i < nr; ++i) {
            if (i == c) continue;
            double f = a[i][c];
            for (int j = 0; j < 2 * nr; ++j) a[i][j] -= f * a[c][j];
        }
    }
    for (int i = 0; i < nr; ++i)
        for (int j = 0; j < nr; ++j) M[i * nr + j] = a[i][nr + j];
}

}  // namespace

void rigid_K_free(int d, int N, const double* rel, const int* body, const int* bfree, const double* Uf, double* out,
                  double sign, cudaStream_t s) {
    ProfScope ps(KID_RIGID_K, s, 0.0);
    k_rigid_K_free<<<grid_1d(N, 128), 128, 0, s>>>(d, N, rel, body, bfree, Uf, out, sign);
    IBR_CHECK_LAUNCH();
}

template <typename Tl>
void rigid_KT_free(int d, int B, const int* bstart, const int* bfree, const double* rel, const Tl* lam, double* out,
                   cudaStream_t s) {
    ProfScope ps(KID_RIGID_KT, s, 0.0);
    k_rigid_KT_free<Tl><<<B, 256, 0, s>>>(d, bstart, bfree, rel, lam, out);
    IBR_CHECK_LAUNCH();
}

template <typename T>
void lam_add_XU(int d, int N, const int* body, const int* bfree, const T* X, const double* Uf, T* lam,
                cudaStream_t s) {
    ProfScope ps(KID_RIGID_K, s, 0.0);
    k_lam_add_XU<T><<<grid_1d((long long)N * d, 128), 128, 0, s>>>(d, N, body, bfree, X, Uf, lam);
    IBR_CHECK_LAUNCH();
}

void body_solve(int nfree, int nr, const double* Nb, const double* r, const double* sv, double* U, cudaStream_t s) {
    ProfScope ps(KID_SMALL, s, 0.0);
    k_body_solve<<<grid_1d(nfree, 32), 32, 0, s>>>(nfree, nr, Nb, r, sv, U);
    IBR_CHECK_LAUNCH();
}

void small_inverse(int nfree, int nr, double* A, int* info, cudaStream_t s) {
    ProfScope ps(KID_SMALL, s, 0.0);
    k_small_inverse<<<grid_1d(nfree, 32), 32, 0, s>>>(nfree, nr, A, info);
    IBR_CHECK_LAUNCH();
}

template void rigid_KT_free<double>(int, int, const int*, const int*, const double*, const double*, double*,
                                    cudaStream_t);
template void rigid_KT_free<float>(int, int, const int*, const int*, const double*, const float*, double*,
                                   cudaStream_t);
template void lam_add_XU<double>(int, int, const int*, const int*, const double*, const double*, double*,
                                 cudaStream_t);
template void lam_add_XU<float>(int, int, const int*, const int*, const float*, const double*, float*, cudaStream_t);

}  // namespace ibr
