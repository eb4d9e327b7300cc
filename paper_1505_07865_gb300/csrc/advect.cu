// Explicit advection of the time-stepped problems (Sec. VII.F, the nozzle):
// N(v) = div(v v) in the centred second-order flux form on the MAC grid, and
// the step forcing g = sigma v^n - rho (c1 N^n + c0 N^{n-1}) + f.
//
// For component a at its face (FP64):
//   N_a = sum_b [F_ab(+1/2) - F_ab(-1/2)] / h
//   F_aa at the cell centres between a-faces: ((v_a(i) + v_a(i+1)) / 2)^2
//   F_ab, b != a, at the edges between a- and b-faces:
//        (v_a averaged along b) * (v_b averaged along a)
// Values beyond a wall come from the App. D extension with the wall data
// (tangential: 2 w - u of the mirror; normal: the wall face holds the wall
// value); wall-face rows get N = 0.  One thread per cell, all components.
#include "ibr_internal.cuh"

namespace ibr {
namespace {

// the field value of component c at (x, y, z), one layer beyond the grid
// allowed on each axis: periodic axes wrap, wall axes use the extension
__device__ double ext_value(const Geo& g, const double* __restrict__ v, const WallData& wd, int c, int x, int y,
                            int z) {
    int id[3] = {x, y, z};
    const int ns[3] = {g.n0, g.n1, g.n2};
    int out_axis = -1;
    for (int a = 0; a < g.d; ++a) {
        if (!((g.wall >> a) & 1)) {
            if (id[a] < 0) id[a] += ns[a];
            if (id[a] >= ns[a]) id[a] -= ns[a];
        } else if (id[a] < 0 || id[a] >= ns[a]) {
            if (out_axis >= 0) return 0.0;  // a wall-wall corner: read by no stencil
            out_axis = a;
        }
    }
    const long long st[3] = {1, ns[0], (long long)ns[0] * ns[1]};
    auto at = [&](int ia) {  // stored value with id[out_axis] replaced by ia
        long long cell = 0;
        for (int e = 0; e < g.d; ++e) cell += (long long)(e == out_axis ? ia : id[e]) * st[e];
        return v[(long long)c * g.ncell + cell];
    };
    auto wall = [&](int a, int side) {  // wall data of component c at this face point
        long long t = 0, s2 = 1;
        for (int e = 0; e < g.d; ++e) {
            if (e == a) continue;
            t += (long long)id[e] * s2;
            s2 *= ns[e];
        }
        const long long nf = g.ncell / ns[a];
        return wd.data[2 * a + side][(long long)c * nf + t];
    };
    // the normal component's stored face 0 lies on the wall: its value is the data
    for (int a = 0; a < g.d; ++a)
        if (((g.wall >> a) & 1) && c == a && a != out_axis && id[a] == 0) return wall(a, 0);
    if (out_axis < 0) return v[(long long)c * g.ncell + id[0] + st[1] * id[1] + st[2] * id[2]];
    const int a = out_axis, n = ns[a], x0 = id[a];
    if (c == a) {  // normal component: faces 0..n, wall faces carry the data
        if (x0 == n) return wall(a, 1);
        if (x0 < 0) return 2.0 * wall(a, 0) - at(-x0);
        return 2.0 * wall(a, 1) - at(2 * n - x0);  // x0 > n: mirror about face n
    }
    if (x0 < 0) return 2.0 * wall(a, 0) - at(-x0 - 1);
    return 2.0 * wall(a, 1) - at(2 * n - 1 - x0);
}

template <int D>
__global__ void __launch_bounds__(256) k_advect(const double* __restrict__ v, double* __restrict__ N, Geo g,
                                                WallData wd, double ih) {
    const int i = blockIdx.x * 32 + threadIdx.x, j = blockIdx.y * 8 + threadIdx.y, k = blockIdx.z;
    if (i >= g.n0 || j >= g.n1) return;
    const long long cell = i + (long long)g.n0 * (j + (long long)g.n1 * k);
    const int id[3] = {i, j, k};
    auto V = [&](int c, int da, int oa, int db, int ob) {  // component c at id + oa e_da + ob e_db
        int p[3] = {id[0], id[1], id[2]};
        p[da] += oa;
        p[db] += ob;
        return ext_value(g, v, wd, c, p[0], p[1], p[2]);
    };
#pragma unroll
    for (int a = 0; a < D; ++a) {
        double acc = 0.0;
        if (((g.wall >> a) & 1) && id[a] == 0) {
            N[(long long)a * g.ncell + cell] = 0.0;
            continue;
        }
#pragma unroll
        for (int b = 0; b < D; ++b) {
            double fp, fm;
            if (b == a) {
                const double u0 = V(a, a, 0, a, 0), up = V(a, a, 1, a, 0), um = V(a, a, -1, a, 0);
                fp = 0.25 * (u0 + up) * (u0 + up);
                fm = 0.25 * (um + u0) * (um + u0);
            } else {
                const double ua_p = 0.5 * (V(a, a, 0, b, 0) + V(a, b, 1, a, 0));
                const double vb_p = 0.5 * (V(b, a, -1, b, 1) + V(b, b, 1, a, 0));
                const double ua_m = 0.5 * (V(a, b, -1, a, 0) + V(a, a, 0, b, 0));
                const double vb_m = 0.5 * (V(b, a, -1, b, 0) + V(b, a, 0, b, 0));
                fp = ua_p * vb_p;
                fm = ua_m * vb_m;
            }
            acc += (fp - fm) * ih;
        }
        N[(long long)a * g.ncell + cell] = acc;
    }
}

__global__ void k_step_force(long long m, const double* __restrict__ v, const double* __restrict__ Nn,
                             const double* __restrict__ Np, const double* __restrict__ f, double sigma, double rc1,
                             double rc0, double* __restrict__ out) {
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= m) return;
    double r = sigma * v[t] - (rc1 * Nn[t] + rc0 * Np[t]);
    if (f) r += f[t];
    out[t] = r;
}

}  // namespace

void advect(const Geo& g, const double* v, const WallData& wd, double* N, cudaStream_t s) {
    dim3 grid((g.n0 + 31) / 32, (g.n1 + 7) / 8, g.n2), blk(32, 8);
    ProfScope ps(KID_ADVECT, s, 2.0 * g.d * g.ncell * sizeof(double));
    if (g.d == 3)
        k_advect<3><<<grid, blk, 0, s>>>(v, N, g, wd, 1.0 / g.h);
    else
        k_advect<2><<<grid, blk, 0, s>>>(v, N, g, wd, 1.0 / g.h);
    IBR_CHECK_LAUNCH();
}

void step_force(long long m, const double* v, const double* Nn, const double* Np, const double* f, double sigma,
                double rho_c1, double rho_c0, double* out, cudaStream_t s) {
    ProfScope ps(KID_AXPBY, s, 5.0 * m * sizeof(double));
    k_step_force<<<grid_1d(m, 256), 256, 0, s>>>(m, v, Nn, Np, f, sigma, rho_c1, rho_c0, out);
    IBR_CHECK_LAUNCH();
}

}  // namespace ibr
