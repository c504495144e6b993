// 27-point stencils of levels whose coefficients do not change along time (every level of
// an extruded design, Sec. 3.4.1) in 2 spatial dimensions.  Row (n, p) of a level operator
// is the sum over the adjacent elements of the masked element-matrix rows: Galerkin blocks
// T_ab on coarse levels (Sec. 3.2), C_e (D_t (x) M_x) + k_e (M_t (x) K_x) on level 0 (Sec.
// 3.1).  Gathered per spatial node p and plane class they form the stencil applied by the
// time-marching kernels (march2d).
#include <math.h>

#include "st_device.cuh"

namespace st {

// class c: 0 first free plane (n = 1 < n_t), 1 interior, 2 last (n = n_t >= 2), 3 n_t == 1.
// The slab below plane n is the first slab (version 0) iff n == 1; the slab above is interior.
template <int LV>
__global__ void k_stencil_build(OpL0<double> o0, OpLc<double> oc, double* __restrict__ out64,
                                float* __restrict__ out32, unsigned char* __restrict__ dir) {
    pdl_enter();
    constexpr int NS = 4, NSYM = 10, NV = 40;
    const Geom& g = LV == 0 ? o0.g : oc.g;
    const long long P = (long long)g.nx1 * g.ny1;
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int i = (int)(p % g.nx1), j = (int)(p / g.nx1);
    dir[p] = sp_dir<2>(g, i, j, 0) ? 1 : 0;
    double F[NV];
    for (int tr = 0; tr < 2; ++tr)
        for (int c = 0; c < 4; ++c) {
            double s[27];
            for (int q = 0; q < 27; ++q) s[q] = 0.0;
            const bool has_above = (c == 0 || c == 1);
            const int slab_below = (c == 0 || c == 3) ? 0 : 1;  // representative slab of its version
            for (int o = 0; o < NS; ++o) {
                const int ex = i - 1 + (o & 1), ey = j - 1 + ((o >> 1) & 1);
                if (ex < 0 || ex >= g.nex || ey < 0 || ey >= g.ney) continue;
                const int as = (~o) & (NS - 1);
                const long long se = (long long)ey * g.nex + ex;
                for (int sb = 0; sb < 2; ++sb) {
                    if (sb == 1 && !has_above) continue;
                    const int at = 1 - sb;
                    const int slab = sb == 0 ? slab_below : 1;
                    if constexpr (LV == 0) {
                        l0_blocks<2>(o0, slab, ex, ey, 0, F);
                    } else {
                        const double* A = oc.elem + elem_index(oc, slab, se) * NV;
                        for (int q = 0; q < NV; ++q) F[q] = A[q];
                    }
                    for (int bt = 0; bt < 2; ++bt) {
                        const int blk = tr ? (bt * 2 + at) : (at * 2 + bt);
                        const int dt = sb + bt;  // plane offset index: 0 (n-1), 1 (n), 2 (n+1)
                        for (int bs = 0; bs < NS; ++bs) {
                            const int di = ex + (bs & 1) - i + 1, dj = ey + ((bs >> 1) & 1) - j + 1;
                            s[dt * 9 + dj * 3 + di] += F[blk * NSYM + symidx<NS>(as, bs)];
                        }
                    }
                }
            }
            for (int q = 0; q < 27; ++q) {
                const long long o = (long long)((tr * 4 + c) * 27 + q) * P + p;
                out64[o] = s[q];
                out32[o] = (float)s[q];
            }
        }
}

// Jacobi diagonal of a stencil level: the centre coefficient (k = 13) of the row's plane class,
// 1 on prescribed rows.  Taken from the stencil itself, so that D is the diagonal of exactly
// the operator the time-marching kernels apply (in FP32 that operator comes from the FP64
// design, not from the BF16 copy the element-wise FP32 rows read).
template <typename T>
__global__ void __launch_bounds__(256) k_stencil_diag(Geom g, const T* __restrict__ coef,
                                                      const unsigned char* __restrict__ dir, T* __restrict__ d,
                                                      int invert) {
    pdl_enter();
    const long long P = (long long)g.nx1 * g.ny1;
    const int nt = g.net;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < g.nnodes;
         q += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(q / P);
        const long long p = q - (long long)n * P;
        T v = T(1);
        if (n > 0 && !dir[p]) {
            const int cls = (n == 1) ? (nt == 1 ? 3 : 0) : (n == nt ? 2 : 1);
            v = coef[((long long)cls * 27 + 13) * P + p];
        }
        d[q] = invert ? T(1) / v : v;
    }
}

template <typename T>
void launch_stencil_diag(const Geom& g, const T* coef, const unsigned char* dir, T* d, bool invert, cudaStream_t s) {
    note_launch(s);
    long long blocks = (g.nnodes + 255) / 256;
    if (blocks > 4 * 1216) blocks = 4 * 1216;
    launch_pdl(k_stencil_diag<T>, (int)(blocks > 0 ? blocks : 1), 256, 0, s, g, coef, dir, d, invert ? 1 : 0);
}
template void launch_stencil_diag<float>(const Geom&, const float*, const unsigned char*, float*, bool, cudaStream_t);
template void launch_stencil_diag<double>(const Geom&, const double*, const unsigned char*, double*, bool,
                                          cudaStream_t);

// Interior rows of a stencil level apply A D^-1 with D^-1 of interior planes, which is the
// same on every interior plane: fold it into the interior-class stencil of both orientations.
// Rows of prescribed spatial nodes become the identity row scaled by their own D^-1.
template <typename T>
__global__ void k_stencil_scale(Geom g, const T* __restrict__ st, const T* __restrict__ dinv,
                                const unsigned char* __restrict__ dir, int nref, T* __restrict__ sc) {
    pdl_enter();
    const long long P = (long long)g.nx1 * g.ny1;
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int i = (int)(p % g.nx1), j = (int)(p / g.nx1);
    const bool pres = dir[p] != 0;
    for (int o = 0; o < 2; ++o)
        for (int k = 0; k < 27; ++k) {
            const int dj = (k % 9) / 3, di = k % 3;
            const int ii = i + di - 1, jn = j + dj - 1;
            const bool ok = ii >= 0 && ii < g.nx1 && jn >= 0 && jn < g.ny1;
            const T c = st[((long long)(o * 4 + 1) * 27 + k) * P + p];
            const T d = ok ? dinv[(long long)nref * P + (long long)jn * g.nx1 + ii] : T(0);
            T v = c * d;
            if (pres) v = k == 13 ? dinv[(long long)nref * P + p] : T(0);
            sc[((long long)o * 27 + k) * P + p] = v;
        }
}

template <typename T>
void launch_stencil_scale(const Geom& g, const T* st, const T* dinv, const unsigned char* dir, T* sc,
                          cudaStream_t s) {
    note_launch(s);
    const long long P = (long long)g.nx1 * g.ny1;
    const int nref = g.net < 2 ? g.net : 2;
    launch_pdl(k_stencil_scale<T>, (int)((P + 127) / 128), 128, 0, s, g, st, dinv, dir, nref, sc);
}
template void launch_stencil_scale<float>(const Geom&, const float*, const float*, const unsigned char*, float*,
                                          cudaStream_t);
template void launch_stencil_scale<double>(const Geom&, const double*, const double*, const unsigned char*, double*,
                                           cudaStream_t);

void launch_stencil_build(int lvl, const OpL0<double>& o0, const OpLc<double>& oc, double* st64, float* st32,
                          unsigned char* dir, cudaStream_t s) {
    note_launch(s);
    const Geom& g = lvl == 0 ? o0.g : oc.g;
    const long long P = (long long)g.nx1 * g.ny1;
    const int blocks = (int)((P + 127) / 128);
    if (lvl == 0)
        launch_pdl(k_stencil_build<0>, blocks, 128, 0, s, o0, oc, st64, st32, dir);
    else
        launch_pdl(k_stencil_build<1>, blocks, 128, 0, s, o0, oc, st64, st32, dir);
}

}  // namespace st
