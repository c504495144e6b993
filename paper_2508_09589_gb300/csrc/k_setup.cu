// Setup-phase kernels: design cast, Galerkin coarse operators J_{l+1} = P^T J_l P
// (arXiv 2508.09589, Sec. 3.2) in element-block form, the dense inverse of the
// coarsest operator, the source vector (Sec. 3.1.2), the p-norm objective and
// its adjoint right-hand side (Sec. 3.3.1, 3.3.3) and the sensitivities (Sec. 3.3.3).
#include <math.h>

#include <mutex>

#include "st_device.cuh"

namespace st {

#define ST_SD_DISPATCH(sd, ...)   \
    do {                          \
        if ((sd) == 2) {          \
            constexpr int SD = 2; \
            __VA_ARGS__;          \
        } else {                  \
            constexpr int SD = 3; \
            __VA_ARGS__;          \
        }                         \
    } while (0)

// Clip the design to [0, 1] and keep FP64 and BF16 copies; a NaN or infinite value sets
// *bad (the caller rejects the design) and is stored as 0.
__global__ void k_design_cast(const double* __restrict__ in, double* __restrict__ g64,
                              __nv_bfloat16* __restrict__ g16, long long n, int* __restrict__ bad) {
    pdl_enter();
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        double v = in[q];
        if (!isfinite(v)) {
            *bad = 1;
            v = 0.0;
        }
        v = v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
        g64[q] = v;
        g16[q] = __double2bfloat16(v);
    }
}

__global__ void k_to_float(const double* __restrict__ in, float* __restrict__ out, long long n) {
    pdl_enter();
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        out[q] = (float)in[q];
}

// One coarse element: A_E = M_E (sum_children Q_c^T A_c Q_c) M_E with Q_c = Q_t (x) Q_s.
template <int SD, int LV>
__global__ void k_build(OpL0<double> f0, OpLc<double> fc, Geom gc, int kind, int tc, double* __restrict__ out) {
    pdl_enter();
    constexpr int NS = 1 << SD, NSYM = NS * (NS + 1) / 2, NV = 4 * NSYM;
    const Geom& gf = LV == 0 ? f0.g : fc.g;
    const long long nstore = tc ? 2 * gc.sp_elems : (long long)gc.net * gc.sp_elems;
    const long long E = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (E >= nstore) return;
    const int N = (int)(E / gc.sp_elems);  // slab (space-time) or version (extruded)
    const long long sec = E - (long long)N * gc.sp_elems;
    double* G = out + E * NV;
    for (int q = 0; q < NV; ++q) G[q] = 0.0;
    if (tc && N == 1 && gc.net < 2) return;
    const int Ex = (int)(sec % gc.nex), Ey = (int)((sec / gc.nex) % gc.ney), Ez = (int)(sec / ((long long)gc.nex * gc.ney));
    const bool cs = kind != 1, ct = kind != 0;
    const int nct = ct ? 2 : 1, ncs = cs ? NS : 1;
    double F[NV];
    double S[4][NS][NS];
    for (int cst = 0; cst < nct; ++cst) {
        const int fslab = ct ? 2 * N + cst : N;
        for (int csp = 0; csp < ncs; ++csp) {
            const int cx = csp & 1, cy = (csp >> 1) & 1, cz = (csp >> 2) & 1;
            const int fx = cs ? 2 * Ex + cx : Ex, fy = cs ? 2 * Ey + cy : Ey;
            const int fz = (SD == 3) ? (cs ? 2 * Ez + cz : Ez) : 0;
            if constexpr (LV == 0) {
                l0_blocks<SD>(f0, fslab, fx, fy, fz, F);
            } else {
                const long long sef = ((long long)fz * gf.ney + fy) * gf.nex + fx;
                const double* A = fc.elem + elem_index(fc, fslab, sef) * NV;
                for (int q = 0; q < NV; ++q) F[q] = A[q];
            }
            // spatial congruence S_ab = Q_s^T F_ab Q_s
            for (int blk = 0; blk < 4; ++blk) {
                for (int i = 0; i < NS; ++i)
                    for (int j = 0; j < NS; ++j) {
                        double acc = 0.0;
                        if (cs) {
                            for (int a = 0; a < NS; ++a) {
                                const double qa = q1(cx + (a & 1), i & 1) * q1(cy + ((a >> 1) & 1), (i >> 1) & 1) *
                                                  (SD == 3 ? q1(cz + ((a >> 2) & 1), (i >> 2) & 1) : 1.0);
                                if (qa == 0.0) continue;
                                for (int b = 0; b < NS; ++b) {
                                    const double qb = q1(cx + (b & 1), j & 1) * q1(cy + ((b >> 1) & 1), (j >> 1) & 1) *
                                                      (SD == 3 ? q1(cz + ((b >> 2) & 1), (j >> 2) & 1) : 1.0);
                                    if (qb == 0.0) continue;
                                    acc += qa * F[blk * NSYM + symidx<NS>(a, b)] * qb;
                                }
                            }
                        } else {
                            acc = F[blk * NSYM + symidx<NS>(i, j)];
                        }
                        S[blk][i][j] = acc;
                    }
            }
            // temporal part: G_cd += sum_ab Qt[a][c] Qt[b][d] S_ab
            for (int c = 0; c < 2; ++c)
                for (int d = 0; d < 2; ++d) {
                    double w[2][2];
                    for (int a = 0; a < 2; ++a)
                        for (int b = 0; b < 2; ++b)
                            w[a][b] = ct ? q1(cst + a, c) * q1(cst + b, d) : ((a == c && b == d) ? 1.0 : 0.0);
                    for (int i = 0; i < NS; ++i)
                        for (int j = i; j < NS; ++j) {
                            double acc = 0.0;
                            for (int a = 0; a < 2; ++a)
                                for (int b = 0; b < 2; ++b)
                                    if (w[a][b] != 0.0) acc += w[a][b] * S[a * 2 + b][i][j];
                            G[(c * 2 + d) * NSYM + symidx<NS>(i, j)] += acc;
                        }
                }
        }
    }
    // coarse masks
    bool fr[2 * NS];
    for (int at = 0; at < 2; ++at)
        for (int as = 0; as < NS; ++as)
            fr[at * NS + as] = (N + at > 0) &&
                               !sp_dir<SD>(gc, Ex + (as & 1), Ey + ((as >> 1) & 1), SD == 3 ? Ez + ((as >> 2) & 1) : 0);
    for (int at = 0; at < 2; ++at)
        for (int bt = 0; bt < 2; ++bt)
            for (int as = 0; as < NS; ++as)
                for (int bs = as; bs < NS; ++bs)
                    if (!(fr[at * NS + as] && fr[bt * NS + bs])) G[(at * 2 + bt) * NSYM + symidx<NS>(as, bs)] = 0.0;
}

// ---------------------------------------------------------------- dense coarsest operator
template <int SD, int LV>
__global__ void k_dense_assemble(OpL0<double> o0, OpLc<double> oc, double* __restrict__ A) {
    pdl_enter();
    constexpr int NS = 1 << SD, NSYM = NS * (NS + 1) / 2, NV = 4 * NSYM;
    const Geom& g = LV == 0 ? o0.g : oc.g;
    const long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long n = g.nnodes;
    if (r >= n) return;
    const int i = (int)(r % g.nx1);
    const int j = (int)((r / g.nx1) % g.ny1);
    const int k = (int)((r / ((long long)g.nx1 * g.ny1)) % g.nz1);
    const int t = (int)(r / g.plane);
    double* row = A + r * n;
    if (!is_free<SD>(g, i, j, k, t)) {
        row[r] = 1.0;
        return;
    }
    double F[NV];
    for (int o = 0; o < NS; ++o) {
        const int ex = i - 1 + (o & 1), ey = j - 1 + ((o >> 1) & 1);
        const int ez = (SD == 3) ? k - 1 + ((o >> 2) & 1) : 0;
        if (ex < 0 || ex >= g.nex || ey < 0 || ey >= g.ney) continue;
        if (SD == 3 && (ez < 0 || ez >= g.nez)) continue;
        const int as = (~o) & (NS - 1);
        const long long se = ((long long)ez * g.ney + ey) * g.nex + ex;
        for (int sb = 0; sb < 2; ++sb) {
            const int slab = t - 1 + sb;
            if (slab < 0 || slab >= g.net) continue;
            const int at = 1 - sb;
            if constexpr (LV == 0) {
                l0_blocks<SD>(o0, slab, ex, ey, ez, F);
            } else {
                const double* E = oc.elem + elem_index(oc, slab, se) * NV;
                for (int q = 0; q < NV; ++q) F[q] = E[q];
            }
            for (int bt = 0; bt < 2; ++bt)
                for (int bs = 0; bs < NS; ++bs) {
                    const int ni = ex + (bs & 1), nj = ey + ((bs >> 1) & 1), nk = SD == 3 ? ez + ((bs >> 2) & 1) : 0;
                    const long long col = (long long)(slab + bt) * g.plane + ((long long)nk * g.ny1 + nj) * g.nx1 + ni;
                    row[col] += F[(at * 2 + bt) * NSYM + symidx<NS>(as, bs)];
                }
        }
    }
}

// One Gauss-Jordan elimination step (no pivoting) from src into dst.  After n steps the
// matrix holds its inverse.  The coarse operators have a positive definite symmetric
// part (the free block) and identity rows at prescribed nodes, so no pivot vanishes.
// pinv[kp] holds 1 / pivot of this step; the thread that writes the next pivot stores its
// reciprocal, so each step needs one division in total.
__global__ void k_gj_first(const double* __restrict__ A, double* __restrict__ pinv, int* err) {
    pdl_enter();
    const double p = A[0];
    if (!(fabs(p) > 1e-300) || !isfinite(p)) *err = 1;
    pinv[0] = (fabs(p) > 1e-300 && isfinite(p)) ? 1.0 / p : 1.0;
}

__global__ void k_gj_step(const double* __restrict__ src, double* __restrict__ dst, int n, int kp,
                          double* __restrict__ pinv, int* err) {
    pdl_enter();
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= (long long)n * n) return;
    const int i = (int)(q / n), j = (int)(q % n);
    const double ip = pinv[kp];
    double v;
    if (i == kp && j == kp)
        v = ip;
    else if (i == kp)
        v = src[(long long)kp * n + j] * ip;
    else if (j == kp)
        v = -src[(long long)i * n + kp] * ip;
    else
        v = src[q] - src[(long long)i * n + kp] * (src[(long long)kp * n + j] * ip);
    dst[q] = v;
    if (i == kp + 1 && j == kp + 1) {
        const bool ok = fabs(v) > 1e-300 && isfinite(v);
        if (!ok) *err = 1;
        pinv[kp + 1] = ok ? 1.0 / v : 1.0;
    }
}

// The whole Gauss-Jordan inverse as ONE cooperative kernel: the n pivot steps are separated by
// a grid barrier instead of a kernel launch each.  Step kp reads the current matrix (src), stages
// its pivot row in shared memory and writes the next one (dst) with the same expression as
// k_gj_step, rows spread over the blocks; the block holding element (kp+1, kp+1) publishes the
// next reciprocal pivot before the barrier.  Every barrier wait is bounded: after `limit` polls
// the kernel sets *tmo and carries on (every loop and index stays bounded whatever the data).
__device__ __forceinline__ void gj_grid_barrier(unsigned* ctr, unsigned target, unsigned limit, int* tmo) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
        unsigned spins = 0;
        while (*((volatile unsigned*)ctr) < target) {
            if (++spins > limit) {
                atomicExch(tmo, 1);
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
    }
    __syncthreads();
}

// Blocked form: BB pivots per step.  With K the step's pivot indices and P = S[K,K]^-1,
// eliminating them one by one is the same as D[K,K] = P, D[K,j] = P S[K,j], D[i,K] = -S[i,K] P
// and D[i,j] = S[i,j] - S[i,K] P S[K,j] (i, j outside K), so a step needs two grid barriers
// (after the new pivot rows, after the update) instead of BB launches.  Every block inverts the
// BB x BB pivot block itself (Gauss-Jordan without pivoting, as the unblocked form); phase 1
// writes the new pivot rows D[K,:] into dst and PR; phase 2 updates the other rows from PR,
// staged in shared memory.
template <int BB>
__global__ void __launch_bounds__(256) k_gj_block(double* A, double* B, double* PR, int n, int* err, unsigned* bar,
                                                  int* tmo, unsigned limit) {
    extern __shared__ double prs[];  // [BB][n] new pivot rows
    __shared__ double Pm[BB][BB];    // inverse of the pivot block
    __shared__ double sik[8][BB];    // S[i, K] of up to 8 rows
    const unsigned nb = gridDim.x;
    unsigned epoch = 0;
    double* src = A;
    double* dst = B;
    for (int kp = 0; kp < n; kp += BB) {
        const int bb = min(BB, n - kp);
        // pivot block inverse: unpivoted Gauss-Jordan on the bb x bb block in shared memory, one
        // thread per entry (the same expression per entry as the unblocked form)
        const int tr = threadIdx.x / BB, tc = threadIdx.x % BB;
        const bool tin = threadIdx.x < BB * BB;
        if (tin) Pm[tr][tc] = (tr < bb && tc < bb) ? __ldcg(src + (long long)(kp + tr) * n + kp + tc) : 0.0;
        __syncthreads();
        for (int k = 0; k < bb; ++k) {
            double v = 0.0;
            if (tin && tr < bb && tc < bb) {
                const double p = Pm[k][k];
                const bool ok = fabs(p) > 1e-300 && isfinite(p);
                if (!ok && tr == k && tc == k && blockIdx.x == 0) *err = 1;
                const double ip = ok ? 1.0 / p : 1.0;
                if (tr == k && tc == k)
                    v = ip;
                else if (tr == k)
                    v = Pm[k][tc] * ip;
                else if (tc == k)
                    v = -Pm[tr][k] * ip;
                else
                    v = Pm[tr][tc] - Pm[tr][k] * (Pm[k][tc] * ip);
            }
            __syncthreads();
            if (tin && tr < bb && tc < bb) Pm[tr][tc] = v;
            __syncthreads();
        }
        // phase 1: new pivot rows D[K, j] = P S[K, j] (j outside K), P (j in K), columns over the grid
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += nb * blockDim.x) {
            double sk[BB];
#pragma unroll
            for (int l = 0; l < BB; ++l) sk[l] = l < bb ? __ldcg(src + (long long)(kp + l) * n + j) : 0.0;
            const bool inK = j >= kp && j < kp + bb;
#pragma unroll
            for (int k = 0; k < BB; ++k) {
                if (k >= bb) break;
                double v;
                if (inK) {
                    v = Pm[k][j - kp];
                } else {
                    v = 0.0;
#pragma unroll
                    for (int l = 0; l < BB; ++l) v += Pm[k][l] * sk[l];
                }
                PR[(long long)k * n + j] = v;
                dst[(long long)(kp + k) * n + j] = v;
            }
        }
        gj_grid_barrier(bar, ++epoch * nb, limit, tmo);
        // phase 2: the other rows, D[i, j] = S[i, j] - S[i, K] PR[:, j]; D[i, K] = -S[i, K] P
        for (int q0 = threadIdx.x; q0 < BB * n; q0 += 8 * blockDim.x) {  // 8 loads in flight per thread
            double t[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int q = q0 + u * blockDim.x;
                t[u] = q < bb * n ? __ldcg(PR + q) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int q = q0 + u * blockDim.x;
                if (q < BB * n) prs[q] = t[u];
            }
        }
        __syncthreads();
        for (int i0 = blockIdx.x; i0 < n; i0 += nb * 8) {
            // up to 8 rows per pass (i0, i0 + nb, ...): their S[i, K] first
            if (threadIdx.x < 8 * BB) {
                const int r = threadIdx.x / BB, l = threadIdx.x % BB, i = i0 + r * nb;
                sik[r][l] = (i < n && l < bb) ? __ldcg(src + (long long)i * n + kp + l) : 0.0;
            }
            __syncthreads();
            for (int r = 0; r < 8; ++r) {
                const int i = i0 + r * nb;
                if (i >= n) break;
                if (i >= kp && i < kp + bb) continue;  // pivot rows were written in phase 1
                const long long row = (long long)i * n;
                double a[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const int j = threadIdx.x + c * 256;
                    a[c] = j < n ? __ldcg(src + row + j) : 0.0;
                }
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const int j = threadIdx.x + c * 256;
                    if (j >= n) break;
                    double v;
                    if (j >= kp && j < kp + bb) {
                        v = 0.0;
#pragma unroll
                        for (int l = 0; l < BB; ++l) v -= sik[r][l] * Pm[l][j - kp];
                    } else {
                        v = a[c];
#pragma unroll
                        for (int l = 0; l < BB; ++l) v -= sik[r][l] * prs[l * n + j];
                    }
                    dst[row + j] = v;
                }
            }
            __syncthreads();
        }
        double* t = src;
        src = dst;
        dst = t;
        gj_grid_barrier(bar, ++epoch * nb, limit, tmo);
    }
}

// ---------------------------------------------------------------- source (Sec. 3.1.2)
// f_i = int N_i Q: spatially uniform Q, so the spatial integral of each adjacent element is
// its volume / 2^SD; the time integral of N_i q(t) over each adjacent slab uses 2-point
// Gauss (exact for uniform q).
template <int SD>
__global__ void k_rhs(Geom g, int kind, double q0, double a, double b, double f, double* __restrict__ out) {
    pdl_enter();
    ST_NODE_LOOP_BEGIN(g)
    double v = 0.0;
    if (is_free<SD>(g, i_, j_, k_, n_)) {
        int nel = 0;
        for (int o = 0; o < (1 << SD); ++o) {
            const int ex = i_ - 1 + (o & 1), ey = j_ - 1 + ((o >> 1) & 1), ez = SD == 3 ? k_ - 1 + ((o >> 2) & 1) : 0;
            if (ex < 0 || ex >= g.nex || ey < 0 || ey >= g.ney) continue;
            if (SD == 3 && (ez < 0 || ez >= g.nez)) continue;
            ++nel;
        }
        double vol = 1.0;
        for (int d = 0; d < SD; ++d) vol *= 0.5 * g.h[d];
        const double xi[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)};
        if (SD == 2 && kind == ST_SRC_GAUSSIAN) {
            // 2-point Gauss per axis in each of the (up to) eight space-time elements of the node:
            // weights (h_x / 2)(h_y / 2)(dt / 2), the node's trilinear basis at each point
            const double cx = 0.5 * g.nex * g.h[0], cy = 0.5 * g.ney * g.h[1];
            const double inv2s2 = 1.0 / (2.0 * a * a);
            for (int o = 0; o < 4; ++o) {
                const int ex = i_ - 1 + (o & 1), ey = j_ - 1 + (o >> 1);
                if (ex < 0 || ex >= g.nex || ey < 0 || ey >= g.ney) continue;
                const int bx = 1 - (o & 1), by = 1 - (o >> 1);  // the node's corner in the element
                for (int sb = 0; sb < 2; ++sb) {
                    const int slab = n_ - 1 + sb;
                    if (slab < 0 || slab >= g.net) continue;
                    const int at = 1 - sb;
                    for (int gt = 0; gt < 2; ++gt) {
                        const double t = (slab + xi[gt]) * g.dt;
                        const double nt_ = at == 1 ? xi[gt] : 1.0 - xi[gt];
                        const double x1 = cx + b * cos(f * t + 0.5 * M_PI), x2 = cy + b * sin(f * t + 0.5 * M_PI);
                        for (int gy = 0; gy < 2; ++gy) {
                            const double y = (ey + xi[gy]) * g.h[1];
                            const double ny_ = by == 1 ? xi[gy] : 1.0 - xi[gy];
                            for (int gx = 0; gx < 2; ++gx) {
                                const double x = (ex + xi[gx]) * g.h[0];
                                const double nx_ = bx == 1 ? xi[gx] : 1.0 - xi[gx];
                                const double r2 = (x - x1) * (x - x1) + (y - x2) * (y - x2);
                                v += vol * 0.5 * g.dt * nx_ * ny_ * nt_ * q0 * exp(-r2 * inv2s2);
                            }
                        }
                    }
                }
            }
        } else {
            double tf = 0.0;
            for (int sb = 0; sb < 2; ++sb) {
                const int slab = n_ - 1 + sb;
                if (slab < 0 || slab >= g.net) continue;
                const int at = 1 - sb;
                for (int gq = 0; gq < 2; ++gq) {
                    const double phi = at == 1 ? xi[gq] : 1.0 - xi[gq];
                    const double t = (slab + xi[gq]) * g.dt;
                    const double q = kind == ST_SRC_SIN_T ? q0 * (a + b * sin(2.0 * M_PI * f * t)) : q0;
                    tf += 0.5 * g.dt * phi * q;
                }
            }
            v = nel * vol * tf;
        }
    }
    out[idx_] = v;
    ST_NODE_LOOP_END
}

// ---------------------------------------------------------------- p-norm objective (Sec. 3.3.1)
template <int SD>
__device__ __forceinline__ double elem_avg(const Geom& g, const double* s, int slab, int ex, int ey, int ez) {
    constexpr int NS = 1 << SD;
    double a = 0.0;
    for (int at = 0; at < 2; ++at)
        for (int bs = 0; bs < NS; ++bs) {
            const int ni = ex + (bs & 1), nj = ey + ((bs >> 1) & 1), nk = SD == 3 ? ez + ((bs >> 2) & 1) : 0;
            a += s[(long long)(slab + at) * g.plane + ((long long)nk * g.ny1 + nj) * g.nx1 + ni];
        }
    return a / (2 * NS);
}

template <int SD>
__global__ void __launch_bounds__(256) k_pnorm_theta(Geom g, const double* __restrict__ s, int P, double* theta,
                                                     RedBuf rb) {
    pdl_enter();
    // element loop: (ex, ey) from the thread grid, (slab, ez) from the plane loop
    double acc[1] = {0.0};
    const int ex = blockIdx.x * blockDim.x + threadIdx.x, ey = blockIdx.y * blockDim.y + threadIdx.y;
    const long long planes = (long long)g.nez * g.net;
    for (long long z = blockIdx.z; z < planes; z += gridDim.z) {
        const int slab = (int)(z / g.nez), ez = (int)(z % g.nez);
        if (ex < g.nex && ey < g.ney) {
            const double T = elem_avg<SD>(g, s, slab, ex, ey, ez);
            acc[0] += ipow(T, P);
        }
    }
    __shared__ double out[1];
    if (reduce_publish<1>(acc, 1, rb, out)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) *theta = out[0];
    }
}

template <int SD>
__global__ void __launch_bounds__(256) k_pnorm_rhs(Geom g, const double* __restrict__ s, int P,
                                                   const double* theta, double* __restrict__ rhs, double* phi) {
    pdl_enter();
    constexpr int NS = 1 << SD;
    const double th = *theta;
    const double sc = pow(th, (1.0 - P) / (double)P) / (2 * NS);
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 && threadIdx.y == 0)
        *phi = pow(th, 1.0 / P);
    ST_NODE_LOOP_BEGIN(g)
    double v = 0.0;
    if (is_free<SD>(g, i_, j_, k_, n_)) {
        for (int o = 0; o < NS; ++o) {
            const int ex = i_ - 1 + (o & 1), ey = j_ - 1 + ((o >> 1) & 1), ez = SD == 3 ? k_ - 1 + ((o >> 2) & 1) : 0;
            if (ex < 0 || ex >= g.nex || ey < 0 || ey >= g.ney) continue;
            if (SD == 3 && (ez < 0 || ez >= g.nez)) continue;
            for (int sb = 0; sb < 2; ++sb) {
                const int slab = n_ - 1 + sb;
                if (slab < 0 || slab >= g.net) continue;
                v += sc * ipow(elem_avg<SD>(g, s, slab, ex, ey, ez), P - 1);
            }
        }
    }
    rhs[idx_] = v;
    ST_NODE_LOOP_END
}

// ---------------------------------------------------------------- sensitivities (Sec. 3.3.3)
// g_e = - Lambda_e^T (C'(gamma_e) (D_t (x) M_x) + k'(gamma_e) (M_t (x) K_x)) s_e; the time
// diffusion k_ad = C dt / 2 scales with C, so it sits in the C' term.  Extruded designs
// accumulate over the slabs of each spatial element in slab order.
template <int SD>
__global__ void k_sens(OpL0<double> op, const double* __restrict__ s, const double* __restrict__ lam,
                       double* __restrict__ out) {
    pdl_enter();
    constexpr int NS = 1 << SD;
    const Geom& g = op.g;
    const long long nout = op.tc ? g.sp_elems : (long long)g.net * g.sp_elems;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= nout) return;
    const long long se = e % g.sp_elems;
    const int ex = (int)(se % g.nex), ey = (int)((se / g.nex) % g.ney), ez = (int)(se / ((long long)g.nex * g.ney));
    const int s0 = op.tc ? 0 : (int)(e / g.sp_elems), s1 = op.tc ? g.net : s0 + 1;
    const double gm = op.g64[e];
    const double dC = op.simp.p_c * op.simp.dC * ipow(gm, op.simp.p_c - 1);
    const double dk = op.simp.p_k * op.simp.dk * ipow(gm, op.simp.p_k - 1);
    const double Dt[2][2] = {{0.0, 0.0}, {-1.0, 1.0}};
    const double Mt[2][2] = {{2.0 * op.dt6, op.dt6}, {op.dt6, 2.0 * op.dt6}};
    long long sidx[NS];
    bool fs[NS];
    for (int bs = 0; bs < NS; ++bs) {
        const int ni = ex + (bs & 1), nj = ey + ((bs >> 1) & 1), nk = SD == 3 ? ez + ((bs >> 2) & 1) : 0;
        sidx[bs] = ((long long)nk * g.ny1 + nj) * g.nx1 + ni;
        fs[bs] = !sp_dir<SD>(g, ni, nj, nk);
    }
    double total = 0.0;
    for (int slab = s0; slab < s1; ++slab) {
        double sv[2][NS], lv[2][NS];
        for (int at = 0; at < 2; ++at)
            for (int bs = 0; bs < NS; ++bs) {
                const bool fr = fs[bs] && (slab + at > 0);
                const long long q = (long long)(slab + at) * g.plane + sidx[bs];
                sv[at][bs] = fr ? s[q] : 0.0;
                lv[at][bs] = fr ? lam[q] : 0.0;
            }
        double acc = 0.0;
        for (int at = 0; at < 2; ++at)
            for (int as = 0; as < NS; ++as) {
                double r = 0.0;
                for (int bt = 0; bt < 2; ++bt)
                    for (int bs = 0; bs < NS; ++bs)
                        r += (dC * Dt[at][bt] * op.mxd[as ^ bs] + dk * Mt[at][bt] * op.kxd[as ^ bs]) * sv[bt][bs];
                acc += lv[at][as] * r;
            }
        total -= acc;
    }
    out[e] = total;
}

// ---------------------------------------------------------------- wrappers
void launch_design_cast(const double* in, double* g64, __nv_bfloat16* g16, long long n, int* bad, cudaStream_t s) {
    note_launch(s);
    const int blocks = (int)((n + 255) / 256 < 65536 ? (n + 255) / 256 : 65536);
    launch_pdl(k_design_cast, blocks > 0 ? blocks : 1, 256, 0, s, in, g64, g16, n, bad);
}

void launch_to_float(const double* in, float* out, long long n, cudaStream_t s) {
    note_launch(s);
    const int blocks = (int)((n + 255) / 256 < 65536 ? (n + 255) / 256 : 65536);
    launch_pdl(k_to_float, blocks > 0 ? blocks : 1, 256, 0, s, in, out, n);
}

void launch_build_from_l0(int sd, const OpL0<double>& f0, const Geom& gc, int kind, int tc, double* elem_c,
                          cudaStream_t s) {
    note_launch(s);
    const long long nstore = tc ? 2 * gc.sp_elems : (long long)gc.net * gc.sp_elems;
    const int blocks = (int)((nstore + 127) / 128);
    OpLc<double> dummy{};
    ST_SD_DISPATCH(sd, launch_pdl(k_build<SD, 0>, blocks, 128, 0, s, f0, dummy, gc, kind, tc, elem_c));
}

void launch_build_from_lc(int sd, const OpLc<double>& fc, const Geom& gc, int kind, double* elem_c, cudaStream_t s) {
    note_launch(s);
    const long long nstore = fc.tc ? 2 * gc.sp_elems : (long long)gc.net * gc.sp_elems;
    const int blocks = (int)((nstore + 127) / 128);
    OpL0<double> dummy{};
    ST_SD_DISPATCH(sd, launch_pdl(k_build<SD, 1>, blocks, 128, 0, s, dummy, fc, gc, kind, fc.tc, elem_c));
}

void launch_dense_assemble(int sd, int lvl, const OpL0<double>& o0, const OpLc<double>& oc, double* A,
                           cudaStream_t s) {
    note_launch(s);
    const Geom& g = lvl == 0 ? o0.g : oc.g;
    cudaMemsetAsync(A, 0, sizeof(double) * g.nnodes * g.nnodes, s);
    const int blocks = (int)((g.nnodes + 127) / 128);
    if (lvl == 0) {
        ST_SD_DISPATCH(sd, launch_pdl(k_dense_assemble<SD, 0>, blocks, 128, 0, s, o0, oc, A));
    } else {
        ST_SD_DISPATCH(sd, launch_pdl(k_dense_assemble<SD, 1>, blocks, 128, 0, s, o0, oc, A));
    }
}

void launch_gauss_jordan(double* A, double* B, double* pinv, double* PR, int n, int* err, unsigned* bar, int* tmo,
                         cudaStream_t s) {
    const long long nn = (long long)n * n;
    // one cooperative launch of the blocked form: a co-resident grid of up to 2 blocks per SM
    if (n <= 4096 && PR) {
        static std::once_flag once;
        // 8 pivots per step (4 when the staged pivot rows, bw n doubles, would not fit in 200 KB);
        // 16 measured no faster on the 1377-node coarsest level of the 256^2 x 256 mesh
        static int per8 = 0, per4 = 0, sms = 0;
        std::call_once(once, [] {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaFuncSetAttribute(k_gj_block<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 8 * 3200 * 8);
            cudaFuncSetAttribute(k_gj_block<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * 4096 * 8);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per8, k_gj_block<8>, 256, 8 * 3200 * 8);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per4, k_gj_block<4>, 256, 4 * 4096 * 8);
        });
        const int bw = n <= 3200 ? 8 : 4;
        const int per = bw == 8 ? per8 : per4;
        int nb = sms * (per < 2 ? per : 2);
        const size_t smem = (size_t)bw * n * sizeof(double);
        if (nb >= 1) {
            cudaMemsetAsync(bar, 0, sizeof(unsigned), s);
            unsigned limit = 1u << 24;  // polls per barrier (about a second) before giving up
            void* args[] = {(void*)&A, (void*)&B, (void*)&PR, (void*)&n, (void*)&err, (void*)&bar, (void*)&tmo,
                            (void*)&limit};
            const void* k = bw == 8 ? (const void*)k_gj_block<8> : (const void*)k_gj_block<4>;
            if (cudaLaunchCooperativeKernel(k, dim3(nb), dim3(256), args, smem, s) == cudaSuccess) {
                note_launch(s);
                const int steps = (n + bw - 1) / bw;
                if (steps & 1) cudaMemcpyAsync(A, B, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s);
                return;
            }
            cudaGetLastError();  // refused (e.g. not co-resident): one launch per pivot below
        }
    }
    note_launch(s, n + 1);
    const int blocks = (int)((nn + 255) / 256);
    double* src = A;
    double* dst = B;
    launch_pdl(k_gj_first, 1, 1, 0, s, A, pinv, err);
    for (int kp = 0; kp < n; ++kp) {
        launch_pdl(k_gj_step, blocks, 256, 0, s, src, dst, n, kp, pinv, err);
        double* t = src;
        src = dst;
        dst = t;
    }
    if (src != A) cudaMemcpyAsync(A, src, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s);
}

void launch_rhs(int sd, const Geom& g, int kind, double q0, double a, double b, double f, double* out,
                cudaStream_t s) {
    note_launch(s);
    const LaunchCfg c = node_cfg(g);
    ST_SD_DISPATCH(sd, launch_pdl(k_rhs<SD>, c.grid, c.block, 0, s, g, kind, q0, a, b, f, out));
}

void launch_pnorm(int sd, const Geom& g, const double* s, int P, double* rhs, double* phi, RedBuf rb,
                  double* scratch, cudaStream_t st) {
    note_launch(st, 2);
    dim3 block(32, 8, 1);
    const int gx = (g.nex + 31) / 32, gy = (g.ney + 7) / 8;
    long long gz = (long long)kMaxBlocks / ((long long)gx * gy);
    const long long planes = (long long)g.nez * g.net;
    if (gz < 1) gz = 1;
    if (gz > planes) gz = planes;
    dim3 grid(gx, gy, (unsigned)gz);
    ST_SD_DISPATCH(sd, launch_pdl(k_pnorm_theta<SD>, grid, block, 0, st, g, s, P, scratch, rb));
    const LaunchCfg c = node_cfg(g);
    ST_SD_DISPATCH(sd, launch_pdl(k_pnorm_rhs<SD>, c.grid, c.block, 0, st, g, s, P, scratch, rhs, phi));
}

void launch_sens(int sd, const OpL0<double>& op, const double* s, const double* lam, double* out, cudaStream_t st) {
    note_launch(st);
    const long long nout = op.tc ? op.g.sp_elems : (long long)op.g.net * op.g.sp_elems;
    const int blocks = (int)((nout + 127) / 128);
    ST_SD_DISPATCH(sd, launch_pdl(k_sens<SD>, blocks, 128, 0, st, op, s, lam, out));
}

}  // namespace st
