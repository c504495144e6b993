// Residual and residual norm of the FP64 fine-level operator for callers that cannot
// allocate device memory (for example code running under another framework's stream
// capture, inside a real-time loop, or with a fixed device-memory pool that forbids
// cudaMalloc).  This is a variant of the FGMRES residual kernel: the same matrix-free
// row evaluation, but its only scratch (one partial sum per thread block and a
// completion counter) lives in the file-scope array below instead of buffers owned by
// a mesh.  Every GPU that loads the library keeps this array until the process exits.
#include <math.h>
#include <string.h>

#include <mutex>

#include "st_device.cuh"

namespace st {

// Maximum number of thread blocks of one call: the x-y plane of the mesh may have at most
// this many 32 x 8 node tiles (for example 1024 x 1024 spatial elements in 2-D space).
constexpr int kNoAllocBlocks = 4096;

// [0, kNoAllocBlocks): per-block partial sums; the next element holds the completion
// counter (its first 4 bytes) and the one after it nothing (padding).
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocBlocks + 2];

namespace {

std::mutex g_na_mu;
void* g_na_ptr[64];  // device address of g_noalloc_scratch per device, set on first use

st_status na_fail(st_status code, const char* msg);

bool na_patch_range(int n, double w, int& lo, int& hi) {
    lo = n + 1;
    hi = -1;
    for (int j = 0; j <= n; ++j)
        if (fabs(2.0 * j - n) <= w * n + 1e-9) {
            lo = j < lo ? j : lo;
            hi = j > hi ? j : hi;
        }
    return true;
}

}  // namespace

// Records a static message for st_last_error without copying it (no host allocation).
st_status set_c_error(st_status code, const char* msg);

namespace {
st_status na_fail(st_status code, const char* msg) { return set_c_error(code, msg); }
}  // namespace

template <int SD>
__global__ void __launch_bounds__(256) k_residual_noalloc(OpL0<double> op, const double* __restrict__ f,
                                                          const double* __restrict__ x, double* __restrict__ r,
                                                          double* __restrict__ norm, double* __restrict__ scratch) {
    const Geom& g = op.g;
    LoadPlain<double, double> ld{x};
    double acc = 0.0;
    ST_NODE_LOOP_BEGIN(g)
    double v;
    if (is_free<SD>(g, i_, j_, k_, n_))
        v = f[idx_] - row_l0<SD, double, false>(op, i_, j_, k_, n_, ld);
    else
        v = f[idx_] - x[idx_];
    r[idx_] = v;
    acc += v * v;
    ST_NODE_LOOP_END
    // block sum, then the last block to finish adds the partials in block order
    __shared__ double sm[32];
    __shared__ int last;
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = (blockDim.x * blockDim.y) >> 5;
#pragma unroll
    for (int off = 16; off; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
    if (lane == 0) sm[warp] = acc;
    __syncthreads();
    const long long bid = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
    const long long nb = (long long)gridDim.x * gridDim.y * gridDim.z;
    unsigned* counter = reinterpret_cast<unsigned*>(scratch + kNoAllocBlocks);
    if (tid == 0) {
        double a = 0;
        for (int w = 0; w < nw; ++w) a += sm[w];
        scratch[bid] = a;
        __threadfence();
        last = atomicAdd(counter, 1u) == (unsigned)(nb - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (warp == 0) {
        double a = 0;
        for (long long b = lane; b < nb; b += 32) a += __ldcg(scratch + b);
#pragma unroll
        for (int off = 16; off; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
        if (lane == 0) {
            *norm = sqrt(a);
            *counter = 0u;  // ready for the next call
        }
    }
}

}  // namespace st

extern "C" st_status st_residual_norm_noalloc(const st_mesh_desc* d, const double* gamma, int layout,
                                              const double* x, const double* f, double* r, double* norm,
                                              void* stream) {
    using namespace st;
    if (!d || !gamma || !x || !f || !r || !norm) return na_fail(ST_ERR_ARG, "null argument");
    const int sd = d->ndim_space;
    if (sd != 2 && sd != 3) return na_fail(ST_ERR_ARG, "ndim_space must be 2 or 3");
    for (int q = 0; q < sd; ++q)
        if (d->n[q] < 1 || !(d->ext[q] > 0)) return na_fail(ST_ERR_ARG, "bad spatial size");
    if (d->n_t < 1 || !(d->tau > 0)) return na_fail(ST_ERR_ARG, "bad time size");
    if (d->mat.p_c < 1 || d->mat.p_k < 1 || d->mat.p_c > 16 || d->mat.p_k > 16)
        return na_fail(ST_ERR_ARG, "SIMP powers must be in [1, 16]");
    if (layout != ST_DESIGN_EXTRUDED && layout != ST_DESIGN_SPACETIME) return na_fail(ST_ERR_ARG, "unknown layout");
    if (d->bc < 0 || d->bc > 3) return na_fail(ST_ERR_ARG, "unknown boundary-condition kind");
    long long nn = d->n_t + 1;
    for (int q = 0; q < sd; ++q) nn *= d->n[q] + 1;
    if (nn > (1LL << 31) - 1) return na_fail(ST_ERR_ARG, "more than 2^31 - 1 nodes");
    const long long tiles = (long long)((d->n[0] + 1 + 31) / 32) * ((d->n[1] + 1 + 7) / 8);
    if (tiles > kNoAllocBlocks)
        return na_fail(ST_ERR_ARG, "x-y plane larger than the static scratch allows (4096 tiles of 32 x 8 nodes)");

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return na_fail(ST_ERR_CUDA, "no current CUDA device");
    }
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!g_na_ptr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return na_fail(ST_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
            }
            g_na_ptr[dev] = p;
        }
        scratch = static_cast<double*>(g_na_ptr[dev]);
    }

    // level-0 geometry and operator tables (host arithmetic only)
    OpL0<double> op{};
    Geom& g = op.g;
    g.nex = d->n[0];
    g.ney = d->n[1];
    g.nez = sd == 3 ? d->n[2] : 1;
    g.net = d->n_t;
    g.nx1 = g.nex + 1;
    g.ny1 = g.ney + 1;
    g.nz1 = sd == 3 ? g.nez + 1 : 1;
    g.nt1 = g.net + 1;
    g.plane = (long long)g.nx1 * g.ny1 * g.nz1;
    g.nnodes = g.plane * g.nt1;
    g.sp_elems = (long long)g.nex * g.ney * g.nez;
    for (int q = 0; q < 3; ++q) g.h[q] = q < sd ? d->ext[q] / d->n[q] : 1.0;
    g.dt = d->tau / d->n_t;
    g.bc = d->bc;
    g.face = d->bc == ST_BC_PATCH_BOTTOM ? 1 : 0;
    for (int q = 0; q < 3; ++q) {
        g.plo[q] = 0;
        g.phi[q] = -1;
    }
    for (int q = 0; q < sd; ++q) na_patch_range(d->n[q], d->bc_width, g.plo[q], g.phi[q]);
    op.g64 = gamma;
    op.g16 = nullptr;
    op.tc = layout == ST_DESIGN_EXTRUDED ? 1 : 0;
    op.simp.C_ins = d->mat.C_ins;
    op.simp.dC = d->mat.C_con - d->mat.C_ins;
    op.simp.k_ins = d->mat.k_ins;
    op.simp.dk = d->mat.k_con - d->mat.k_ins;
    op.simp.p_c = d->mat.p_c;
    op.simp.p_k = d->mat.p_k;
    const int NS = 1 << sd;
    for (int mb = 0; mb < 8; ++mb) {
        double mx = 0.0, kx = 0.0;
        if (mb < NS) {
            mx = 1.0;
            for (int dd = 0; dd < sd; ++dd) mx *= ((mb >> dd) & 1) ? g.h[dd] / 6.0 : g.h[dd] / 3.0;
            for (int dd = 0; dd < sd; ++dd) {
                double t = ((mb >> dd) & 1) ? -1.0 / g.h[dd] : 1.0 / g.h[dd];
                for (int e = 0; e < sd; ++e)
                    if (e != dd) t *= ((mb >> e) & 1) ? g.h[e] / 6.0 : g.h[e] / 3.0;
                kx += t;
            }
        }
        op.mxd[mb] = mx;
        op.kxd[mb] = kx;
    }
    op.dt6 = g.dt / 6.0;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the completion counter must start at zero (a previous call that failed mid-way may
    // have left it set); the partial sums are overwritten by every call
    if (cudaMemsetAsync(scratch + kNoAllocBlocks, 0, sizeof(unsigned), s) != cudaSuccess) {
        cudaGetLastError();
        return na_fail(ST_ERR_CUDA, "clearing the static scratch failed");
    }
    const LaunchCfg c = node_cfg(g);
    if ((long long)c.grid.x * c.grid.y * c.grid.z > kNoAllocBlocks) return na_fail(ST_ERR_ARG, "grid too large");
    if (sd == 2)
        k_residual_noalloc<2><<<c.grid, c.block, 0, s>>>(op, f, x, r, norm, scratch);
    else
        k_residual_noalloc<3><<<c.grid, c.block, 0, s>>>(op, f, x, r, norm, scratch);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(ST_ERR_CUDA, "kernel launch failed");
    note_launch(s);
    return ST_OK;
}
