// PDE filter and Heaviside projection of the design (Sec. 3.3.2).  The filter solves the
// reaction-diffusion equation -div(D grad psi) + psi = gamma over the space-time domain, D =
// diag(r_x^2/12 per spatial axis, r_t^2/12 in time), natural boundary conditions, discretised
// with the trilinear (16-node in 3+1-D) space-time elements of the mesh: (M_f + K_f) psi = T
// gamma, T_ie = v_e / n_v, and the filtered element value is the mean of its nodal values.
// The matrix has constant coefficients, a tensor product of 1-D mass and stiffness matrices,
// so row i depends only on whether node i lies on the lower boundary, inside or on the upper
// boundary along each axis: its 3^(SD+1) coefficients come from a table of 3^(SD+1) classes.
// The system is SPD and solved by Jacobi-preconditioned conjugate gradients.
#include <math.h>

#include "st_device.cuh"

namespace st {

// class of a node along an axis with n elements: 0 lower boundary, 1 interior, 2 upper boundary
__device__ __forceinline__ int fclass(int i, int n) { return i == 0 ? 0 : (i == n ? 2 : 1); }

// y = A x, or (dinv != null) the Jacobi inverse diagonal.  tab[class][offset], offsets in
// order (t, [z,] y, x) with x fastest, each in {-1, 0, 1}.
template <int SD>
__global__ void __launch_bounds__(256) k_filter_apply(Geom g, const double* __restrict__ tab, const double* __restrict__ x,
                                                      double* __restrict__ y, double* __restrict__ dinv) {
    pdl_enter();
    constexpr int NO = SD == 2 ? 27 : 81;
    ST_NODE_LOOP_BEGIN(g)
    const int ct = fclass(n_, g.net), cz = SD == 3 ? fclass(k_, g.nez) : 0, cy = fclass(j_, g.ney), cx = fclass(i_, g.nex);
    const int cls = SD == 2 ? (ct * 3 + cy) * 3 + cx : ((ct * 3 + cz) * 3 + cy) * 3 + cx;
    const double* c = tab + (long long)cls * NO;
    if (dinv) {
        dinv[idx_] = 1.0 / c[NO / 2];
    } else {
        double acc = 0.0;
#pragma unroll
        for (int o = 0; o < NO; ++o) {
            const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1;
            const int oz = SD == 3 ? (o / 9) % 3 - 1 : 0;
            const int ot = SD == 3 ? o / 27 - 1 : o / 9 - 1;
            if ((ox < 0 && cx == 0) || (ox > 0 && cx == 2) || (oy < 0 && cy == 0) || (oy > 0 && cy == 2)) continue;
            if (SD == 3 && ((oz < 0 && cz == 0) || (oz > 0 && cz == 2))) continue;
            if ((ot < 0 && ct == 0) || (ot > 0 && ct == 2)) continue;
            const long long q = idx_ + ox + (long long)oy * g.nx1 + (long long)oz * g.nx1 * g.ny1 + (long long)ot * g.plane;
            acc += c[o] * x[q];
        }
        y[idx_] = acc;
    }
    ST_NODE_LOOP_END
}

// nodal right-hand side (T gamma)_i = scale * sum of the values of the elements around node i
template <int SD>
__global__ void __launch_bounds__(256) k_filter_rhs(Geom g, const double* __restrict__ gam, double scale,
                                                    double* __restrict__ out) {
    pdl_enter();
    ST_NODE_LOOP_BEGIN(g)
    double acc = 0.0;
    for (int o = 0; o < (1 << (SD + 1)); ++o) {
        const int ex = i_ - 1 + (o & 1), ey = j_ - 1 + ((o >> 1) & 1);
        const int ez = SD == 3 ? k_ - 1 + ((o >> 2) & 1) : 0;
        const int et = n_ - 1 + ((o >> SD) & 1);
        if (ex < 0 || ex >= g.nex || ey < 0 || ey >= g.ney || et < 0 || et >= g.net) continue;
        if (SD == 3 && (ez < 0 || ez >= g.nez)) continue;
        acc += gam[(((long long)et * g.nez + ez) * g.ney + ey) * g.nex + ex];
    }
    out[idx_] = acc * scale;
    ST_NODE_LOOP_END
}

// element means of a nodal field
template <int SD>
__global__ void __launch_bounds__(256) k_filter_mean(Geom g, const double* __restrict__ psi, double* __restrict__ out) {
    pdl_enter();
    const long long ne = g.sp_elems * g.net;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x) {
        long long r = e;
        const int ex = (int)(r % g.nex);
        r /= g.nex;
        const int ey = (int)(r % g.ney);
        r /= g.ney;
        const int ez = SD == 3 ? (int)(r % g.nez) : 0;
        if (SD == 3) r /= g.nez;
        const int et = (int)r;
        double acc = 0.0;
        for (int a = 0; a < (1 << (SD + 1)); ++a) {
            const int i = ex + (a & 1), j = ey + ((a >> 1) & 1), k = SD == 3 ? ez + ((a >> 2) & 1) : 0;
            const int n = et + ((a >> SD) & 1);
            acc += psi[(((long long)n * g.nz1 + k) * g.ny1 + j) * g.nx1 + i];
        }
        out[e] = acc / (double)(1 << (SD + 1));
    }
}

// conjugate-gradient updates: x += a p, r -= a q;  z = D^-1 r, p = z + b p;  p = z + b p
__global__ void __launch_bounds__(256) k_cg_xr(long long n, double a, const double* __restrict__ p,
                                               const double* __restrict__ q, double* __restrict__ x,
                                               double* __restrict__ r) {
    pdl_enter();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        x[i] += a * p[i];
        r[i] -= a * q[i];
    }
}
__global__ void __launch_bounds__(256) k_cg_zp(long long n, double b, const double* __restrict__ dinv,
                                               const double* __restrict__ r, double* z, double* p) {
    pdl_enter();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double zi = dinv[i] * r[i];
        const double pi = p[i];
        z[i] = zi;
        p[i] = zi + b * pi;
    }
}
__global__ void __launch_bounds__(256) k_cg_p(long long n, double b, const double* __restrict__ z, double* __restrict__ p) {
    pdl_enter();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = z[i] + b * p[i];
}

// projection H and its derivative, element by element
__global__ void __launch_bounds__(256) k_heaviside(long long n, const double* __restrict__ in, double* __restrict__ out,
                                                   double* __restrict__ dout, double beta, double eta) {
    pdl_enter();
    const double den = tanh(beta * eta) + tanh(beta * (1.0 - eta));
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double t = tanh(beta * (in[i] - eta));
        if (out) out[i] = (tanh(beta * eta) + t) / den;
        if (dout) dout[i] = beta * (1.0 - t * t) / den;
    }
}

static int flat_blocks(long long n) {
    long long b = (n + 255) / 256;
    if (b > 4 * 1216) b = 4 * 1216;
    return (int)(b > 0 ? b : 1);
}

void launch_filter_apply(int sd, const Geom& g, const double* tab, const double* x, double* y, double* dinv,
                         cudaStream_t s) {
    note_launch(s);
    const LaunchCfg c = node_cfg(g);
    if (sd == 2)
        launch_pdl(k_filter_apply<2>, c.grid, c.block, 0, s, g, tab, x, y, dinv);
    else
        launch_pdl(k_filter_apply<3>, c.grid, c.block, 0, s, g, tab, x, y, dinv);
}
void launch_filter_rhs(int sd, const Geom& g, const double* gam, double scale, double* out, cudaStream_t s) {
    note_launch(s);
    const LaunchCfg c = node_cfg(g);
    if (sd == 2)
        launch_pdl(k_filter_rhs<2>, c.grid, c.block, 0, s, g, gam, scale, out);
    else
        launch_pdl(k_filter_rhs<3>, c.grid, c.block, 0, s, g, gam, scale, out);
}
void launch_filter_mean(int sd, const Geom& g, const double* psi, double* out, cudaStream_t s) {
    note_launch(s);
    const int b = flat_blocks(g.sp_elems * g.net);
    if (sd == 2)
        launch_pdl(k_filter_mean<2>, b, 256, 0, s, g, psi, out);
    else
        launch_pdl(k_filter_mean<3>, b, 256, 0, s, g, psi, out);
}
void launch_cg_xr(long long n, double a, const double* p, const double* q, double* x, double* r, cudaStream_t s) {
    note_launch(s);
    launch_pdl(k_cg_xr, flat_blocks(n), 256, 0, s, n, a, p, q, x, r);
}
void launch_cg_zp(long long n, double b, const double* dinv, const double* r, double* z, double* p, cudaStream_t s) {
    note_launch(s);
    launch_pdl(k_cg_zp, flat_blocks(n), 256, 0, s, n, b, dinv, r, z, p);
}
void launch_cg_p(long long n, double b, const double* z, double* p, cudaStream_t s) {
    note_launch(s);
    launch_pdl(k_cg_p, flat_blocks(n), 256, 0, s, n, b, z, p);
}
void launch_heaviside(long long n, const double* in, double* out, double* dout, double beta, double eta,
                      cudaStream_t s) {
    note_launch(s);
    launch_pdl(k_heaviside, flat_blocks(n), 256, 0, s, n, in, out, dout, beta, eta);
}

}  // namespace st
