// Coarse-level rows of space-time 2-D designs (FP32 multigrid) as time-marching kernels, on the
// levels reached from level 0 by coarsening space only.  There the Galerkin product keeps the
// fine time matrices: the block of slab s and coarse element e is D_t (x) M_se + M_t (x) K_se,
// D_t = [[0, 0], [-1, 1]], M_t = dt/6 [[2, 1], [1, 2]] (Sec. 2.2's factorisation, summed over the
// fine elements with the spatial interpolation), so each (slab, element) carries two 4 x 4
// spatial matrices.  They are extracted once per design (k_x2_blocks) from the FP64 blocks and
// stored in FP32 as full rows, [slab][element][M rows 0..3, K rows 0..3]: each corner node of
// an element reads its own two rows, so every stored value is read once per apply.
//
// Slab s couples planes s and s + 1.  With SM_b = M_se[a] x_b and SK_b = K_se[a] x_b (the node at
// corner a of element e, x_b the element's four values on plane s + b), slab s adds to
//   A:   row s (a_t = 0):     dt/3 SK_0 + dt/6 SK_1,          row s + 1 (a_t = 1): -SM_0 + dt/6 SK_0 + SM_1 + dt/3 SK_1
//   A^T: row s:               dt/3 SK_0 - SM_1 + dt/6 SK_1,   row s + 1:           dt/6 SK_0 + SM_1 + dt/3 SK_1
// summed over the four elements around the node.  The first slab's blocks have the t = 0 rows
// and columns removed; only its block (1, 1) reaches a free row, so it is stored as M = block
// (1, 1), K = 0.  Prescribed neighbours contribute nothing (x is masked); prescribed rows are
// the identity.
//
// A block owns a 32 x 8 tile and a chunk of time planes.  Per plane, the input vectors' halo
// rows are staged by cp.async in 16-byte chunks into a ring PF planes ahead and x is formed in
// place (as in k_l0st.cu); each thread gathers its 3 x 3 neighbourhood of plane m, applies
// slab m - 1 with the neighbourhood of plane m - 1 kept in registers, and loads the rows of
// slab m for the next plane.  Modes as in k_l0st.cu:
//   0: w = A D^-1 u, 1: r = b - A x, 2: u_0 = b - A x and ||u_0||^2, 3: y = A x.
#include <mutex>

#include "k_ring.cuh"

namespace st {

namespace {

struct LcstRing {
    static constexpr int VW = 4;               // floats per chunk
    static constexpr int ROWC = 10, ROW = 40;  // chunks / staged floats per halo row (34 cells, any offset)
    static constexpr int PLANE = 10 * ROW;
    static constexpr int NCH = 10 * ROWC;
    static constexpr int PF = 8, RING = PF + 1;
    static constexpr int NPAIR = PLANE / 2;
};

template <int NQ>
struct LcstLayout {
    using R = LcstRing;
    static constexpr unsigned PLANEB = R::PLANE * 4;
    static constexpr unsigned SLOTB = NQ * PLANEB;
    static constexpr size_t smem = (size_t)R::RING * SLOTB;
};

}  // namespace

template <int MODE, bool TR>
__global__ void __launch_bounds__(256, 2) km_lcst(Geom g, const float* __restrict__ blk, float dt, int chunk,
                                                  const float* __restrict__ u, const float* __restrict__ dinv,
                                                  const float* __restrict__ b, float* __restrict__ out, int j,
                                                  int steps, SmState* st_, RedBuf rb) {
    pdl_enter();
    using R = LcstRing;
    constexpr int NQ = MODE == 0 ? 2 : 1;
    using LY = LcstLayout<NQ>;
    constexpr int ROW = R::ROW, ROWC = R::ROWC, M = R::VW - 1, PF = R::PF, RING = R::RING;
    constexpr unsigned PLANEB = LY::PLANEB, SLOTB = LY::SLOTB, ROWB = ROW * 4;
    if constexpr (MODE == 0) {
        const SmStateT<float>* st = smt<float>(st_);
        if (st->stop || j >= st->kdim) return;
    }
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 8;
    const int i = i0 + tx, jj = j0 + ty;
    const int nt = g.net, nx1 = g.nx1, ny1 = g.ny1, nex = g.nex, ney = g.ney;
    const int n0 = blockIdx.z * chunk;
    const int n1 = min(n0 + chunk, nt + 1);
    const int ms = n0 > 0 ? n0 - 1 : 0;
    const int me = n1 <= nt ? n1 : nt;
    const int P = (int)g.plane;
    const int N = (int)g.nnodes;
    const int SP = (int)g.sp_elems;
    const bool in = i < nx1 && jj < ny1;
    const int p = in ? jj * nx1 + i : 0;
    const bool dirp = in ? sp_dir<2>(g, i, jj, 0) : true;
    const unsigned cwin = (unsigned)__cvta_generic_to_shared(g_step_smem);
    const float dt3 = dt / 3.f, dt6 = dt / 6.f;

    // copy role: threads < NQ NCH, a chunk position of one staged vector
    const bool cvec = tid < NQ * R::NCH;
    const int cv = cvec ? tid / R::NCH : 0;
    const int cpos = cvec ? tid - cv * R::NCH : 0;
    const int ccy = cpos / ROWC, cch = cpos - ccy * ROWC;
    const int cgy = j0 - 1 + ccy;
    const bool crow = cvec && cgy >= 0 && cgy < ny1;
    const int crowE = cgy * nx1 + (i0 - 1);
    const unsigned cdst = cwin + (unsigned)cv * PLANEB + 4u * (unsigned)(ccy * ROW + cch * R::VW);
    const float* csrc = cv == 0 ? u : dinv;
    // x-forming role: the element pair at ue of halo row uy (threads < NPAIR)
    const bool uthr = tid < R::NPAIR;
    const int uy = uthr ? tid / (ROW / 2) : 0;
    const int ue = uthr ? 2 * (tid - uy * (ROW / 2)) : 0;
    const int urowE = (j0 - 1 + uy) * nx1 + (i0 - 1);
    const unsigned usrc = 4u * (unsigned)(uy * ROW + ue);
    const int uroff = urowE & M;
    unsigned umask = 0;
#pragma unroll
    for (int sh = 0; sh <= M; ++sh)
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const int ci = i0 - 1 + ue + l - sh, cj = j0 - 1 + uy;
            if (ci >= 0 && ci < nx1 && cj >= 0 && cj < ny1 && sp_dir<2>(g, ci, cj, 0)) umask |= 1u << (2 * sh + l);
        }
    int roff[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) roff[d] = ((j0 - 1 + ty + d) * nx1 + (i0 - 1)) & M;
    const unsigned gbase = 4u * (unsigned)(ty * ROW + tx);
    // the four elements o around the node: their index in a slab (or -1) and the node's corner
    int eidx[4];
#pragma unroll
    for (int o = 0; o < 4; ++o) {
        const int ex = i - 1 + (o & 1), ey = jj - 1 + (o >> 1);
        eidx[o] = (in && ex >= 0 && ex < nex && ey >= 0 && ey < ney) ? ey * nex + ex : -1;
    }

    auto issue = [&](int m, int k) {
        if (cvec && m <= me) {
            const int E = m * P + crowE;
            const int A = (E & ~M) + cch * R::VW;
            int bytes = crow ? 16 : 0;
            if (m == 0 || m == nt) {
                bytes = 0;
                if (crow && A >= 0 && A < N) bytes = A <= N - R::VW ? 16 : (N - A) * 4;
            }
            cp_async16(cdst + (unsigned)k * SLOTB, csrc + (bytes ? A : 0), bytes);
        }
        cp_async_commit();
    };
    auto form_x = [&](int m, int k) {
        if (!uthr) return;
        const unsigned a = usrc + (unsigned)k * SLOTB;
        float x0, x1;
        lds2<float>(a, x0, x1);
        if constexpr (NQ == 2) {
            float d0, d1;
            lds2<float>(a + PLANEB, d0, d1);
            x0 *= d0;
            x1 *= d1;
        }
        const unsigned o = m == 0 ? 3u : (umask >> (2 * ((m * P + uroff) & M))) & 3u;
        if (o & 1u) x0 = 0.f;
        if (o & 2u) x1 = 0.f;
        sts2<float>(a, x0, x1);
    };
    // rows of slab s of the four elements: corner (3 - o) rows of M and K
    auto load_slab = [&](int s, float4 (&Mr)[4], float4 (&Kr)[4]) {
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            if (eidx[o] >= 0 && s >= 0 && s < nt) {
                const float4* e = reinterpret_cast<const float4*>(blk + ((long long)s * SP + eidx[o]) * 32);
                Mr[o] = __ldg(e + (3 - o));
                Kr[o] = __ldg(e + 4 + (3 - o));
            } else {
                Mr[o] = make_float4(0.f, 0.f, 0.f, 0.f);
                Kr[o] = Mr[o];
            }
        }
    };
    float nrm = 0.f;
    auto emit = [&](int r, float a) {
        const int qn = r * P + p;
        float v = a;
        if (r == 0 || dirp) v = MODE == 0 ? u[qn] * dinv[qn] : u[qn];
        if constexpr (MODE == 0 || MODE == 3) {
            out[qn] = v;
        } else {
            const float rr = b[qn] - v;
            out[qn] = rr;
            if constexpr (MODE == 2) nrm += rr * rr;
        }
    };

#pragma unroll 1
    for (int d = 0; d < PF; ++d) issue(ms + d, d);
    cp_async_wait<PF - 1>();
    __syncthreads();
    form_x(ms, 0);
    float4 Mc[4], Kc[4];  // slab m - 1 at plane m
    load_slab(ms, Mc, Kc);
    float xp[9];          // plane m - 1 neighbourhood
    float aT = 0.f;       // row m: the top part of slab m - 1
    int km = 0;
#pragma unroll 1
    for (int m = ms; m <= me; ++m) {
        cp_async_wait<PF - 2>();
        __syncthreads();
        const int k1 = km + 1 == RING ? 0 : km + 1;
        issue(m + PF, km == 0 ? RING - 1 : km - 1);
        if (m + 1 <= me) form_x(m + 1, k1);
        float4 Mn[4], Kn[4];
        if (m > ms) load_slab(m, Mn, Kn);  // slab m, for the next plane
        const int mp = (m * P) & M;
        const unsigned base = gbase + (unsigned)km * SLOTB;
        const unsigned r0 = base + 4u * (unsigned)((mp + roff[0]) & M);
        const unsigned r1 = base + ROWB + 4u * (unsigned)((mp + roff[1]) & M);
        const unsigned r2 = base + 2 * ROWB + 4u * (unsigned)((mp + roff[2]) & M);
        float xc[9];
        xc[0] = lds1<float>(r0), xc[1] = lds1<float>(r0 + 4), xc[2] = lds1<float>(r0 + 8);
        xc[3] = lds1<float>(r1), xc[4] = lds1<float>(r1 + 4), xc[5] = lds1<float>(r1 + 8);
        xc[6] = lds1<float>(r2), xc[7] = lds1<float>(r2 + 4), xc[8] = lds1<float>(r2 + 8);
        if (m > ms) {
            // slab m - 1: planes m - 1 (xp) and m (xc)
            float sm0 = 0.f, sk0 = 0.f, sm1 = 0.f, sk1 = 0.f;
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int ox = o & 1, oy = o >> 1;
                // the element's nodes b = 0..3 (x bit, y bit) in the neighbourhood
                const int c0 = oy * 3 + ox, c1 = c0 + 1, c2 = c0 + 3, c3 = c0 + 4;
                sm0 += Mc[o].x * xp[c0] + Mc[o].y * xp[c1] + Mc[o].z * xp[c2] + Mc[o].w * xp[c3];
                sk0 += Kc[o].x * xp[c0] + Kc[o].y * xp[c1] + Kc[o].z * xp[c2] + Kc[o].w * xp[c3];
                sm1 += Mc[o].x * xc[c0] + Mc[o].y * xc[c1] + Mc[o].z * xc[c2] + Mc[o].w * xc[c3];
                sk1 += Kc[o].x * xc[c0] + Kc[o].y * xc[c1] + Kc[o].z * xc[c2] + Kc[o].w * xc[c3];
            }
            float bot, top;
            if constexpr (!TR) {
                bot = dt3 * sk0 + dt6 * sk1;
                top = (sm1 - sm0) + dt6 * sk0 + dt3 * sk1;
            } else {
                bot = dt3 * sk0 - sm1 + dt6 * sk1;
                top = dt6 * sk0 + sm1 + dt3 * sk1;
            }
            if (in && m - 1 >= n0 && m - 1 < n1) emit(m - 1, aT + bot);
            aT = top;
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                Mc[o] = Mn[o];
                Kc[o] = Kn[o];
            }
        }
        if (in && m == nt && nt >= n0 && nt < n1) emit(nt, aT);
#pragma unroll
        for (int q = 0; q < 9; ++q) xp[q] = xc[q];
        km = k1;
    }
    cp_async_wait<0>();
    if constexpr (MODE == 2) {
        float acc[1] = {nrm};
        __shared__ double red_out[1];
        if (reduce_publish_t<float, 1>(acc, 1, rb, red_out)) {
            if (tid == 0) sm_start_finish<float>(st_, red_out[0], steps);
        }
    }
}

namespace {
template <int MODE, bool TR>
void launch_lcst_t(const OpLc<float>& op, const float* u, const float* dinv, const float* b, float* out, int j,
                   int steps, SmState* st, RedBuf rb, cudaStream_t s) {
    dim3 grid, block;
    const MarchGrid mg = march_grid(op.g, grid, block);
    constexpr size_t bytes = LcstLayout<MODE == 0 ? 2 : 1>::smem;
    static std::once_flag attr;
    std::call_once(attr, [] {
        cudaFuncSetAttribute(km_lcst<MODE, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    });
    launch_pdl(km_lcst<MODE, TR>, grid, block, bytes, s, op.g, op.x2blk, (float)op.g.dt, mg.chunk, u, dinv, b, out,
               j, steps, st, rb);
}
}  // namespace

bool lcst_usable(const OpLc<float>& op, const void* const* vecs, int nvec) {
    if (op.x2blk == nullptr || op.g.nz1 != 1) return false;
    if (op.g.nnodes > (1LL << 31) - 64 || op.g.plane < 64) return false;
    for (int q = 0; q < nvec; ++q)
        if (vecs[q] && ((uintptr_t)vecs[q] & 15u) != 0) return false;
    return true;
}

void launch_lcst(int mode, bool tr, const OpLc<float>& op, const float* u, const float* dinv, const float* b,
                 float* out, int j, int steps, SmState* st, RedBuf rb, cudaStream_t s) {
    if (mode == 0)
        tr ? launch_lcst_t<0, true>(op, u, dinv, b, out, j, steps, st, rb, s)
           : launch_lcst_t<0, false>(op, u, dinv, b, out, j, steps, st, rb, s);
    else if (mode == 1)
        tr ? launch_lcst_t<1, true>(op, u, dinv, b, out, j, steps, st, rb, s)
           : launch_lcst_t<1, false>(op, u, dinv, b, out, j, steps, st, rb, s);
    else if (mode == 2)
        tr ? launch_lcst_t<2, true>(op, u, dinv, b, out, j, steps, st, rb, s)
           : launch_lcst_t<2, false>(op, u, dinv, b, out, j, steps, st, rb, s);
    else
        tr ? launch_lcst_t<3, true>(op, u, dinv, b, out, j, steps, st, rb, s)
           : launch_lcst_t<3, false>(op, u, dinv, b, out, j, steps, st, rb, s);
}

// M and K of every (slab, element) of a space-coarsened level of a space-time 2-D design, in FP64
// from the level's FP64 blocks, as full FP32 rows: slab s >= 1: K = 3/dt block (0, 0),
// M = block (1, 1) - block (0, 0); slab 0 (t = 0 removed): M = block (1, 1), K = 0.
__global__ void __launch_bounds__(256) k_x2_blocks(OpLc<double> op, double dt, float* __restrict__ out) {
    const Geom& g = op.g;
    const long long ne = (long long)g.net * g.sp_elems;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= ne) return;
    constexpr int NS = 4, NSYM = 10, NV = 4 * NSYM;
    const int slab = (int)(e / g.sp_elems);
    const double* A = op.elem + e * NV;  // per-slab storage: element index slab * sp_elems + se
    float* o = out + e * 32;
    for (int a = 0; a < NS; ++a)
        for (int bn = 0; bn < NS; ++bn) {
            const double f00 = A[0 * NSYM + symidx<NS>(a, bn)], f11 = A[3 * NSYM + symidx<NS>(a, bn)];
            const double k = slab > 0 ? 3.0 / dt * f00 : 0.0;
            const double mm = slab > 0 ? f11 - f00 : f11;
            o[a * 4 + bn] = (float)mm;
            o[16 + a * 4 + bn] = (float)k;
        }
}

void launch_x2_blocks(const OpLc<double>& op, float* out, cudaStream_t s) {
    const long long ne = (long long)op.g.net * op.g.sp_elems;
    k_x2_blocks<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(op, op.g.dt, out);
}

}  // namespace st
