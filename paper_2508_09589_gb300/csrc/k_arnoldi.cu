// Fused Arnoldi step of the Jacobi-GMRES smoother (Sec. 3.2) for levels applied as
// 27-point time-marching stencils (extruded designs, 2 spatial dimensions), FP32.
//
// Step j -> j+1 in one pass:
//   u_{j+1} = s_j w_j - sum_{q<=j} c_q u_q          (c_q = H[q][j] s_q, known)
//   w_{j+1} = A D^{-1} u_{j+1}                      (stencil on the freshly formed vector)
//   ||u_{j+1}||^2 and (w_{j+1}, u_q), q <= j+1       (one reduction)
// u_{j+1} is formed on the tile and its halo (the halo recomputed by each block), so the
// update and the apply share one read of the basis instead of two.  The raw operands of
// a plane (w_j, u_0..u_j, dinv at the thread's staging cells) arrive by cp.async into a
// per-thread shared-memory ring PF planes ahead; each thread consumes only the cells it
// staged itself, so the ring needs no block barrier.
#include <math.h>

#include <mutex>

#include "st_device.cuh"

namespace st {

constexpr int kArnPF = 2;  // planes in flight

// Dynamic shared memory layout (floats): raw[kArnPF][NQ + 1][2][256] (slot 0: w_j,
// slots 1..j+1: u_0..u_j, slot NQ: dinv; per thread two staging cells), then
// tileX[2][10][34] (D^{-1} u_{j+1} with halo), then tileU[2][NQ][8][32] (u_0..u_{j+1} of
// the interior cells).
template <int NQ>
struct ArnSmem {
    static constexpr int raw = kArnPF * (NQ + 1) * 2 * 256;
    static constexpr int tileX = 2 * 10 * 34;
    static constexpr int tileU = 2 * NQ * 8 * 32;
    static constexpr int floats = raw + tileX + tileU;
};

template <int NQ>
__global__ void __launch_bounds__(256) km_arnoldi(Geom g, const float* __restrict__ coef,
                                                  const unsigned char* __restrict__ dir, int chunk,
                                                  const float* __restrict__ dinv, Ptrs<float> U,
                                                  const float* __restrict__ w_in, float* __restrict__ w_out, int j,
                                                  SmState* st_, RedBuf rb) {
    pdl_enter();
    const SmStateT<float>* st = smt<float>((const SmState*)st_);
    if (st->stop || j >= st->kdim) return;
    extern __shared__ float sm[];
    float* raw = sm;
    float(*tileX)[10][34] = reinterpret_cast<float(*)[10][34]>(sm + ArnSmem<NQ>::raw);
    float(*tileU)[NQ][8][32] = reinterpret_cast<float(*)[NQ][8][32]>(sm + ArnSmem<NQ>::raw + ArnSmem<NQ>::tileX);
    __shared__ float cf[NQ];
    __shared__ float sj_s;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    if (tid <= j) cf[tid] = st->H[tid * kMaxSmooth + j] * st->s[tid];
    if (tid == 0) sj_s = st->s[j];
    __syncthreads();
    const float sj = sj_s;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 8;
    const int i = i0 + tx, jj = j0 + ty;
    const int n0 = blockIdx.z * chunk;
    const int n1 = min(n0 + chunk, g.nt1);
    const long long P = (long long)g.nx1 * g.ny1;
    const bool in = i < g.nx1 && jj < g.ny1;
    const long long p = in ? (long long)jj * g.nx1 + i : 0;
    const int nt = g.net;
    float* const un = U.p[j + 1];

    // this thread's two staging cells of the 34 x 10 tile (+ halo)
    long long cell_off[2];
    bool cell_ok[2], cell_st[2], cell_int[2];
    int cell_sy[2], cell_sx[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int cidx = tid + r * 256;
        cell_off[r] = 0;
        cell_ok[r] = false;
        cell_st[r] = cidx < 340;
        cell_int[r] = false;
        cell_sy[r] = 0;
        cell_sx[r] = 0;
        if (cidx < 340) {
            const int cy = cidx / 34, cx = cidx - cy * 34;
            cell_sy[r] = cy;
            cell_sx[r] = cx;
            const int gi = i0 - 1 + cx, gj = j0 - 1 + cy;
            if (gi >= 0 && gi < g.nx1 && gj >= 0 && gj < g.ny1) {
                cell_off[r] = (long long)gj * g.nx1 + gi;
                cell_ok[r] = true;
                cell_int[r] = cx >= 1 && cx <= 32 && cy >= 1 && cy <= 8;
            }
        }
    }
    // raw slot address for (ring stage s, operand k, cell r): per-thread private
    auto rawp = [&](int s, int k, int r) -> float* { return raw + (((s * (NQ + 1) + k) * 2 + r) * 256 + tid); };
    auto issue = [&](int n, int s) {
        const bool okn = n >= 0 && n <= nt;
        const long long base = (long long)(n < 0 ? 0 : (n > nt ? nt : n)) * P;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            if (!cell_st[r]) continue;
            const bool v = okn && cell_ok[r];
            const long long q = base + cell_off[r];
            cp_async4(rawp(s, 0, r), w_in + q, v);
#pragma unroll
            for (int k = 0; k < NQ - 1; ++k)
                if (k <= j) cp_async4(rawp(s, 1 + k, r), U.p[k] + q, v);
            cp_async4(rawp(s, NQ, r), dinv + q, v);
        }
        cp_async_commit();
    };

    float c[27];
#pragma unroll
    for (int q = 0; q < 27; ++q) c[q] = in ? coef[(long long)(27 + q) * P + p] : 0.f;
    const bool dirp = in ? (dir[p] != 0) : true;

    float acc[NQ + 1];  // [0]: ||u_{j+1}||^2, [1 + q]: (w_{j+1}, u_q)
#pragma unroll
    for (int q = 0; q <= NQ; ++q) acc[q] = 0.f;

    int buf = 0;
    // form u_{j+1} at this thread's cells of plane n (raw ring stage s), stage D^{-1} u_{j+1}
    // into tileX[buf] and u_0..u_{j+1} of interior cells into tileU[buf], write u_{j+1}
    // for owned cells, then read this thread's neighbourhood and own basis values.
    auto stage = [&](int n, int s, float (&dst9)[9], float (&own)[NQ]) {
        cp_async_wait<kArnPF - 1>();
        const bool okn = n >= 0 && n <= nt;
        const bool owned = n >= n0 && n < n1;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            if (!cell_st[r]) continue;
            float v = sj * *rawp(s, 0, r);
#pragma unroll
            for (int k = 0; k < NQ - 1; ++k)
                if (k <= j) v -= cf[k] * *rawp(s, 1 + k, r);
            const bool valid = okn && cell_ok[r];
            v = valid ? v : 0.f;
            tileX[buf][cell_sy[r]][cell_sx[r]] = v * *rawp(s, NQ, r);
            if (cell_int[r]) {
                const int ly = cell_sy[r] - 1, lx = cell_sx[r] - 1;
#pragma unroll
                for (int k = 0; k < NQ - 1; ++k)
                    if (k <= j) tileU[buf][k][ly][lx] = *rawp(s, 1 + k, r);
                tileU[buf][j + 1][ly][lx] = v;
                if (owned && valid) {
                    un[(long long)n * P + cell_off[r]] = v;
                    acc[0] += v * v;
                }
            }
        }
        issue(n + kArnPF, s);  // refill this stage (only this thread reads it)
        __syncthreads();
#pragma unroll
        for (int dj = 0; dj < 3; ++dj)
#pragma unroll
            for (int di = 0; di < 3; ++di) dst9[dj * 3 + di] = tileX[buf][ty + dj][tx + di];
#pragma unroll
        for (int k = 0; k < NQ; ++k) own[k] = k <= j + 1 ? tileU[buf][k][ty][tx] : 0.f;
        buf ^= 1;
    };
    auto row = [&](int n, const float (&xa)[9], const float (&xb)[9], const float (&xc)[9], const float (&own)[NQ]) {
        if (!in) return;
        float y;
        if (n == 0 || dirp) {
            y = xb[4];
        } else {
            const int cls = (n == 1) ? (nt == 1 ? 3 : 0) : (n == nt ? 2 : 1);
            float a0 = 0, a1 = 0, a2 = 0;
            if (cls == 1) {
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    a0 += c[k] * xa[k];
                    a1 += c[9 + k] * xb[k];
                    a2 += c[18 + k] * xc[k];
                }
            } else {
                const float* cc = coef + (long long)cls * 27 * P + p;
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    a0 += cc[(long long)k * P] * xa[k];
                    a1 += cc[(long long)(9 + k) * P] * xb[k];
                    a2 += cc[(long long)(18 + k) * P] * xc[k];
                }
            }
            y = a0 + a1 + a2;
        }
        w_out[(long long)n * P + p] = y;
#pragma unroll
        for (int k = 0; k < NQ; ++k)
            if (k <= j + 1) acc[1 + k] += y * own[k];
    };

    // prologue: ring stages hold planes n0-1, n0 (stage 0, 1); window and own values of
    // planes n0-1 and n0; then the loop stages plane n+1 while computing row n.
    float x0[9], x1[9], x2[9];
    float o0[NQ], o1[NQ], o2[NQ];
    issue(n0 - 1, 0);
    issue(n0, 1);
    stage(n0 - 1, 0, x0, o0);
    stage(n0, 1, x1, o1);
    int s = 0;  // ring stage holding plane n + 1
    for (int n = n0; n < n1; n += 3) {
        stage(n + 1, s, x2, o2);
        s ^= 1;
        row(n, x0, x1, x2, o1);
        if (n + 1 < n1) {
            stage(n + 2, s, x0, o0);
            s ^= 1;
            row(n + 1, x1, x2, x0, o2);
        }
        if (n + 2 < n1) {
            stage(n + 3, s, x1, o1);
            s ^= 1;
            row(n + 2, x2, x0, x1, o0);
        }
    }
    cp_async_wait<0>();

    __shared__ double out[NQ + 1];
    if (reduce_publish_t<float, NQ + 1>(acc, j + 3, rb, out)) {
        if (tid == 0) {
            SmStateT<float>* S = smt<float>(st_);
            const float h = (float)sqrt(out[0]);
            S->H[(j + 1) * kMaxSmooth + j] = h;
            sm_givens_column_t<float>(S, j);
            const bool brk = !(h > 1e-6f * S->beta) || !isfinite(h);
            if (brk) {
                S->kdim = j + 1;
                sm_backsolve_t<float>(S, j + 1);
            } else {
                const float s1 = 1.f / h;
                S->s[j + 1] = s1;
                for (int q = 0; q <= j + 1; ++q) S->H[q * kMaxSmooth + j + 1] = S->s[q] * s1 * (float)out[1 + q];
            }
        }
    }
}

template <int NQ>
static void launch_arnoldi_nq(const Geom& g, const float* coef, const unsigned char* dir, const float* dinv,
                              const Ptrs<float>& U, const float* w_in, float* w_out, int j, SmState* st, RedBuf rb,
                              cudaStream_t s) {
    dim3 grid, block;
    const MarchGrid mg = march_grid(g, grid, block);
    const size_t bytes = sizeof(float) * ArnSmem<NQ>::floats;
    // once per process (the server's slot threads reach this concurrently)
    static std::once_flag attr;
    std::call_once(attr, [&] {
        cudaFuncSetAttribute(km_arnoldi<NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    });
    launch_pdl(km_arnoldi<NQ>, grid, block, bytes, s, g, coef, dir, mg.chunk, dinv, U, w_in, w_out, j, st, rb);
}

// One fused Arnoldi step j -> j+1 (requires j + 2 <= 16).
void launch_arnoldi(const Geom& g, const float* coef, const unsigned char* dir, const float* dinv,
                    const Ptrs<float>& U, const float* w_in, float* w_out, int j, SmState* st, RedBuf rb,
                    cudaStream_t s) {
    note_launch(s);
    if (j + 2 <= 4)
        launch_arnoldi_nq<4>(g, coef, dir, dinv, U, w_in, w_out, j, st, rb, s);
    else if (j + 2 <= 8)
        launch_arnoldi_nq<8>(g, coef, dir, dinv, U, w_in, w_out, j, st, rb, s);
    else
        launch_arnoldi_nq<16>(g, coef, dir, dinv, U, w_in, w_out, j, st, rb, s);
}

}  // namespace st
