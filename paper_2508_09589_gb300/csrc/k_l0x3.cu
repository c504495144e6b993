// Operator rows for extruded (time-constant) designs in three space dimensions (FP32
// multigrid), as time-marching kernels, on level 0 and on the coarse levels.  With the design
// constant in time, every element block of a level is a Kronecker sum D_t (x) M_e + M_t (x) K_e
// (Sec. 2.2's factorisation on level 0, C_e M_x and k_e K_x; Galerkin products of it on coarse
// levels, where the 2 x 2 time matrices D_t and M_t of the level come from the nested linear
// interpolation in time), so each node's row is a combination of two time-constant 27-point
// spatial stencils: MC = sum_e M_e and KD = sum_e K_e over the eight elements around it.  With
// sM = MC x_q and sK = KD x_q on plane q, T_ab = D_t[a][b] sM + M_t[a][b] sK and e_s = 1 when
// slab s exists (0 <= s < n_t), plane q adds to the rows it touches:
//   A:   row q + 1: e_q T_10,   row q: e_{q-1} T_11 + e_q T_00,   row q - 1: e_{q-1} T_01
//   A^T: row q + 1: e_q T_01,   row q: (the same),                row q - 1: e_{q-1} T_10
// (on level 0: D_t = [[0, 0], [-1, 1]], M_t = [[2, 1], [1, 2]] with dt/6 folded into KD).
// Prescribed neighbours (the t = 0 plane and the spatial Dirichlet set) contribute nothing;
// prescribed rows are the identity.
//
// A block owns a 16 x 4 x 4 tile of spatial nodes and a chunk of time planes; each thread
// holds its node's two stencils for the whole march: on level 0 built from the BF16 design of
// the eight elements around it, on coarse levels read from the stencils extracted once per
// design (k_x3_stencil).  Per plane, the 36 halo rows (18 x 6 x 6 cells) of the input vectors
// are staged by cp.async as the 16-byte chunks that cover them into a ring PF planes ahead; one
// pass forms x (u D^-1 in the smoother, masked at prescribed cells) into a double-buffered
// plane at fixed positions; each thread reads its 27 neighbours from it.  Modes as in
// k_l0st.cu:
//   0: w = A D^-1 u, 1: r = b - A x, 2: u_0 = b - A x and ||u_0||^2, 3: y = A x.
#include <mutex>

#include "k_ring.cuh"

namespace st {

namespace {

struct L0x3Ring {
    static constexpr int TX = 16, TY = 4, TZ = 4;  // tile of spatial nodes
    static constexpr int HX = TX + 2, HY = TY + 2, HZ = TZ + 2;
    static constexpr int NROW = HY * HZ;           // halo rows (along x) per plane
    static constexpr int VW = 4;                   // floats per chunk
    static constexpr int ROWC = (VW - 1 + HX + VW - 1) / VW, ROW = ROWC * VW;  // 6 chunks, 24 floats
    static constexpr int PLANE = NROW * ROW;       // staged floats of one vector-plane
    static constexpr int NCH = NROW * ROWC;        // chunk positions per vector-plane
    static constexpr int NX = NROW * HX;           // cells of the formed x plane
    static constexpr int PF = 8, RING = PF;        // planes in flight; plane m's slot is refilled once x_m is formed
};

template <int NQ>
struct L0x3Layout {
    using R = L0x3Ring;
    static constexpr unsigned PLANEB = R::PLANE * 4;
    static constexpr unsigned SLOTB = NQ * PLANEB;
    static constexpr unsigned XB0 = R::RING * SLOTB;  // two formed x planes after the ring
    static constexpr unsigned XPB = R::NX * 4;
    static constexpr size_t smem = (size_t)XB0 + 2 * XPB;
    static_assert(SLOTB % 16 == 0, "slots start on 16-byte boundaries");
};

constexpr int kCopyUnits = 2;  // copy units per thread (NQ NCH <= 512)
constexpr int kXUnits = 3;     // x cells per thread (NX <= 768)

}  // namespace

// What the marching kernel reads of a level: its geometry; on level 0 the BF16 design, SIMP
// laws and the Q1 tables (M_x, K_x by a ^ b; dt/6); on coarse levels the extracted stencils
// [54][P] (MC, then KD); the level's time matrices D_t, M_t ([a_t][b_t], row-major).
struct X3Op {
    Geom g;
    const __nv_bfloat16* g16;
    Simp simp;
    float mxd[8], kxd[8], dt6;
    const float* st;
    float tw[8];
};

template <int MODE, bool TR, bool L0>
__global__ void __launch_bounds__(256, 2) km_l0x3(X3Op op, int chunk, int gyt, const float* __restrict__ u,
                                                  const float* __restrict__ dinv, const float* __restrict__ b,
                                                  float* __restrict__ out, int j, int steps, SmState* st_,
                                                  RedBuf rb) {
    pdl_enter();
    using R = L0x3Ring;
    constexpr int NQ = MODE == 0 ? 2 : 1;
    using LY = L0x3Layout<NQ>;
    constexpr int M = R::VW - 1, PF = R::PF, RING = R::RING;
    constexpr unsigned PLANEB = LY::PLANEB, SLOTB = LY::SLOTB;
    static_assert(NQ * R::NCH <= 256 * kCopyUnits && R::NX <= 256 * kXUnits, "units per thread");
    if constexpr (MODE == 0) {
        const SmStateT<float>* st = smt<float>(st_);
        if (st->stop || j >= st->kdim) return;
    }
    const Geom& g = op.g;
    const int t = threadIdx.x;
    const int tx = t & 15, ty = (t >> 4) & 3, tz = t >> 6;
    const int i0 = blockIdx.x * R::TX, j0 = (blockIdx.y % gyt) * R::TY, k0 = (blockIdx.y / gyt) * R::TZ;
    const int i = i0 + tx, jj = j0 + ty, kk = k0 + tz;
    const int nt = g.net, nx1 = g.nx1, ny1 = g.ny1, nz1 = g.nz1;
    const int n0 = blockIdx.z * chunk;
    const int n1 = min(n0 + chunk, nt + 1);
    const int ms = n0 > 0 ? n0 - 1 : 0;
    const int me = n1 <= nt ? n1 : nt;
    const int P = (int)g.plane;
    const int N = (int)g.nnodes;
    const bool in = i < nx1 && jj < ny1 && kk < nz1;
    const int p = in ? (kk * ny1 + jj) * nx1 + i : 0;
    const bool dirp = in ? sp_dir<3>(g, i, jj, kk) : true;
    const unsigned cwin = (unsigned)__cvta_generic_to_shared(g_step_smem);

    // the node's two stencils: on level 0 from the eight elements around it (BF16 design,
    // constant in time), on coarse levels from the extracted stencils
    float MC[27], KD[27];
#pragma unroll
    for (int q = 0; q < 27; ++q) MC[q] = KD[q] = 0.f;
    if (!L0 && in) {
#pragma unroll
        for (int q = 0; q < 27; ++q) {
            MC[q] = op.st[(long long)q * P + p];
            KD[q] = op.st[(long long)(27 + q) * P + p];
        }
    }
    if (L0 && in) {
        const float cins = (float)op.simp.C_ins, cd = (float)op.simp.dC, kins = (float)op.simp.k_ins,
                    kd = (float)op.simp.dk;
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            const int ox = o & 1, oy = (o >> 1) & 1, oz = o >> 2;
            const int ex = i - 1 + ox, ey = jj - 1 + oy, ez = kk - 1 + oz;
            if (ex < 0 || ex >= g.nex || ey < 0 || ey >= g.ney || ez < 0 || ez >= g.nez) continue;
            const float gm = __bfloat162float(op.g16[(ez * g.ney + ey) * g.nex + ex]);
            const float c = cins + cd * ipow(gm, op.simp.p_c);
            const float dk = op.dt6 * (kins + kd * ipow(gm, op.simp.p_k));
            const int as = (~o) & 7;
#pragma unroll
            for (int bn = 0; bn < 8; ++bn) {
                const int q = ((oz + (bn >> 2)) * 3 + oy + ((bn >> 1) & 1)) * 3 + ox + (bn & 1);
                MC[q] += c * op.mxd[as ^ bn];
                KD[q] += dk * op.kxd[as ^ bn];
            }
        }
    }

    // copy units: (vector, chunk position) pairs, unit c = t + 256 r
    int cE[kCopyUnits], cch_[kCopyUnits];
    unsigned cdst[kCopyUnits];
    bool cok[kCopyUnits], crow[kCopyUnits];
    const float* csrc[kCopyUnits];
#pragma unroll
    for (int r = 0; r < kCopyUnits; ++r) {
        const int c = t + 256 * r;
        cok[r] = c < NQ * R::NCH;
        const int v = cok[r] ? c / R::NCH : 0;
        const int pos = cok[r] ? c - v * R::NCH : 0;
        const int rr = pos / R::ROWC, ch = pos - rr * R::ROWC;
        const int ry = rr % R::HY, rz = rr / R::HY;
        const int gj = j0 - 1 + ry, gk = k0 - 1 + rz;
        crow[r] = cok[r] && gj >= 0 && gj < ny1 && gk >= 0 && gk < nz1;
        cE[r] = (gk * ny1 + gj) * nx1 + (i0 - 1);
        cch_[r] = ch;
        cdst[r] = cwin + (unsigned)v * PLANEB + 4u * (unsigned)(rr * R::ROW + ch * R::VW);
        csrc[r] = v == 0 ? u : dinv;
    }
    // x units: cell c = t + 256 r of the formed plane (row rr, column cx), its row's element
    // offset on plane 0 and whether the cell is prescribed
    int xsrc[kXUnits], xroff[kXUnits];
    unsigned xdst[kXUnits], xmask[kXUnits];
    bool xok[kXUnits];
#pragma unroll
    for (int r = 0; r < kXUnits; ++r) {
        const int c = t + 256 * r;
        xok[r] = c < R::NX;
        const int rr = xok[r] ? c / R::HX : 0, cx = xok[r] ? c - rr * R::HX : 0;
        const int ry = rr % R::HY, rz = rr / R::HY;
        const int gi = i0 - 1 + cx, gj = j0 - 1 + ry, gk = k0 - 1 + rz;
        xroff[r] = ((gk * ny1 + gj) * nx1 + (i0 - 1)) & M;
        xsrc[r] = rr * R::ROW + cx;
        xdst[r] = 4u * (unsigned)c;
        const bool inside = gi >= 0 && gi < nx1 && gj >= 0 && gj < ny1 && gk >= 0 && gk < nz1;
        xmask[r] = (inside && sp_dir<3>(g, gi, gj, gk)) ? 1u : 0u;
    }
    const unsigned gbase = 4u * (unsigned)((tz * R::HY + ty) * R::HX + tx);  // neighbour (0, 0, 0)

    auto issue = [&](int m, int k) {
        if (m <= me) {
#pragma unroll
            for (int r = 0; r < kCopyUnits; ++r) {
                if (!cok[r]) continue;
                const int E = m * P + cE[r];
                const int A = (E & ~M) + cch_[r] * R::VW;
                int bytes = crow[r] ? 16 : 0;
                if (m == 0 || m == nt) {  // the chunk may begin before the vector or run past its end
                    bytes = 0;
                    if (crow[r] && A >= 0 && A < N) bytes = A <= N - R::VW ? 16 : (N - A) * 4;
                }
                cp_async16(cdst[r] + (unsigned)k * SLOTB, csrc[r] + (bytes ? A : 0), bytes);
            }
        }
        cp_async_commit();
    };
    // x of plane m (ring slot k) into formed plane buffer xb
    auto form_x = [&](int m, int k, int xb) {
        const int mp = (m * P) & M;
#pragma unroll
        for (int r = 0; r < kXUnits; ++r) {
            if (!xok[r]) continue;
            const unsigned a = (unsigned)k * SLOTB + 4u * (unsigned)(xsrc[r] + ((mp + xroff[r]) & M));
            float x = lds1<float>(a);
            if constexpr (NQ == 2) x *= lds1<float>(a + PLANEB);
            if (m == 0 || xmask[r]) x = 0.f;
            *reinterpret_cast<float*>(g_step_smem + LY::XB0 + (unsigned)xb * LY::XPB + xdst[r]) = x;
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
    cp_async_wait<PF - 1>();  // plane ms
    __syncthreads();
    form_x(ms, 0, ms & 1);
    float aP = 0.f, aC = 0.f;
    int km = 0;
#pragma unroll 1
    for (int m = ms; m <= me; ++m) {
        cp_async_wait<PF - 2>();  // plane m + 1
        __syncthreads();
        const int k1 = km + 1 == RING ? 0 : km + 1;
        issue(m + PF, km);  // plane m's slot: x_m is formed
        if (m + 1 <= me) form_x(m + 1, k1, (m + 1) & 1);
        const unsigned xbase = LY::XB0 + (unsigned)(m & 1) * LY::XPB + gbase;
        float sM = 0.f, sK = 0.f;
#pragma unroll
        for (int dz = 0; dz < 3; ++dz)
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    const int q = (dz * 3 + dy) * 3 + dx;
                    const float v = lds1<float>(xbase + 4u * (unsigned)((dz * R::HY + dy) * R::HX + dx));
                    sM += MC[q] * v;
                    sK += KD[q] * v;
                }
        const float eq = m < nt ? 1.f : 0.f, eq1 = m >= 1 ? 1.f : 0.f;
        const float t00 = op.tw[0] * sM + op.tw[4] * sK, t01 = op.tw[1] * sM + op.tw[5] * sK;
        const float t10 = op.tw[2] * sM + op.tw[6] * sK, t11 = op.tw[3] * sM + op.tw[7] * sK;
        const float aN = eq * (TR ? t01 : t10);
        aP += eq1 * (TR ? t10 : t01);
        aC += eq1 * t11 + eq * t00;
        if (in && m - 1 >= n0 && m - 1 < n1) emit(m - 1, aP);
        if (in && m == nt && nt >= n0 && nt < n1) emit(nt, aC);
        aP = aC;
        aC = aN;
        km = k1;
    }
    cp_async_wait<0>();
    if constexpr (MODE == 2) {
        float acc[1] = {nrm};
        __shared__ double red_out[1];
        if (reduce_publish_t<float, 1>(acc, 1, rb, red_out)) {
            if (t == 0) sm_start_finish<float>(st_, red_out[0], steps);
        }
    }
}

namespace {
template <int MODE, bool TR, bool L0>
void launch_x3_t(const X3Op& op, const float* u, const float* dinv, const float* b, float* out, int j, int steps,
                 SmState* st, RedBuf rb, cudaStream_t s) {
    using R = L0x3Ring;
    const Geom& g = op.g;
    const int gx = (g.nx1 + R::TX - 1) / R::TX, gyt = (g.ny1 + R::TY - 1) / R::TY, gzt = (g.nz1 + R::TZ - 1) / R::TZ;
    const long long tiles = (long long)gx * gyt * gzt;
    const long long budget = g.march_blocks > 0 && g.march_blocks < kMaxBlocks ? g.march_blocks : kMarchBlocks;
    long long gz = budget / tiles;
    if (gz < 1) gz = 1;
    if (gz > g.nt1) gz = g.nt1;
    const int chunk = (int)((g.nt1 + gz - 1) / gz);
    gz = (g.nt1 + chunk - 1) / chunk;
    constexpr size_t bytes = L0x3Layout<MODE == 0 ? 2 : 1>::smem;
    static std::once_flag attr;
    std::call_once(attr, [] {
        cudaFuncSetAttribute(km_l0x3<MODE, TR, L0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    });
    launch_pdl(km_l0x3<MODE, TR, L0>, dim3((unsigned)gx, (unsigned)(gyt * gzt), (unsigned)gz), dim3(256), bytes, s,
               op, chunk, gyt, u, dinv, b, out, j, steps, st, rb);
}

template <bool L0>
void launch_x3(int mode, bool tr, const X3Op& op, const float* u, const float* dinv, const float* b, float* out,
               int j, int steps, SmState* st, RedBuf rb, cudaStream_t s) {
    if (mode == 0)
        tr ? launch_x3_t<0, true, L0>(op, u, dinv, b, out, j, steps, st, rb, s)
           : launch_x3_t<0, false, L0>(op, u, dinv, b, out, j, steps, st, rb, s);
    else if (mode == 1)
        tr ? launch_x3_t<1, true, L0>(op, u, dinv, b, out, j, steps, st, rb, s)
           : launch_x3_t<1, false, L0>(op, u, dinv, b, out, j, steps, st, rb, s);
    else if (mode == 2)
        tr ? launch_x3_t<2, true, L0>(op, u, dinv, b, out, j, steps, st, rb, s)
           : launch_x3_t<2, false, L0>(op, u, dinv, b, out, j, steps, st, rb, s);
    else
        tr ? launch_x3_t<3, true, L0>(op, u, dinv, b, out, j, steps, st, rb, s)
           : launch_x3_t<3, false, L0>(op, u, dinv, b, out, j, steps, st, rb, s);
}

bool vecs_aligned(const void* const* vecs, int nvec) {
    for (int q = 0; q < nvec; ++q)
        if (vecs[q] && ((uintptr_t)vecs[q] & 15u) != 0) return false;
    return true;
}

bool x3_geom_usable(const Geom& g) {
    if (g.nz1 <= 1 || g.nnodes > (1LL << 31) - 64) return false;
    if (g.plane < 64) return false;  // the chunks of a plane's last halo row end inside the next plane
    const long long gyz = (long long)((g.ny1 + 3) / 4) * ((g.nz1 + 3) / 4);
    return gyz <= 65535;  // grid.y
}
}  // namespace

bool l0x3_usable(const OpL0<float>& op, const void* const* vecs, int nvec) {
    if (!op.tc || op.g16 == nullptr) return false;  // extruded 3-D designs only
    return x3_geom_usable(op.g) && vecs_aligned(vecs, nvec);
}

void launch_l0x3(int mode, bool tr, const OpL0<float>& op, const float* u, const float* dinv, const float* b,
                 float* out, int j, int steps, SmState* st, RedBuf rb, cudaStream_t s) {
    X3Op x{};
    x.g = op.g;
    x.g16 = op.g16;
    x.simp = op.simp;
    for (int q = 0; q < 8; ++q) {
        x.mxd[q] = op.mxd[q];
        x.kxd[q] = op.kxd[q];
    }
    x.dt6 = op.dt6;
    const float tw[8] = {0.f, 0.f, -1.f, 1.f, 2.f, 1.f, 1.f, 2.f};  // D_t, and M_t with dt/6 in KD
    for (int q = 0; q < 8; ++q) x.tw[q] = tw[q];
    launch_x3<true>(mode, tr, x, u, dinv, b, out, j, steps, st, rb, s);
}

bool lcx3_usable(const OpLc<float>& op, const void* const* vecs, int nvec) {
    return op.x3st != nullptr && x3_geom_usable(op.g) && vecs_aligned(vecs, nvec);
}

void launch_lcx3(int mode, bool tr, const OpLc<float>& op, const float* u, const float* dinv, const float* b,
                 float* out, int j, int steps, SmState* st, RedBuf rb, cudaStream_t s) {
    X3Op x{};
    x.g = op.g;
    x.st = op.x3st;
    for (int q = 0; q < 8; ++q) x.tw[q] = op.x3tw[q];
    launch_x3<false>(mode, tr, x, u, dinv, b, out, j, steps, st, rb, s);
}

// The two stencils of every node of a coarse level of an extruded 3-D design, in FP64 from the
// level's FP64 element blocks F[a_t b_t] = D_t[a_t][b_t] M_e + M_t[a_t][b_t] K_e (the version of
// the slabs after the first): M_e and K_e row a of each element from the blocks (0, 0) and
// (1, 1), summed over the eight elements around the node; rounded to FP32, [54][P].
__global__ void __launch_bounds__(256) k_x3_stencil(OpLc<double> op, double d00, double d11, double m00,
                                                    double m11, float* __restrict__ out) {
    const Geom& g = op.g;
    const long long P = g.plane;
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int i = (int)(p % g.nx1), jj = (int)((p / g.nx1) % g.ny1), kk = (int)(p / ((long long)g.nx1 * g.ny1));
    constexpr int NS = 8, NSYM = NS * (NS + 1) / 2, NV = 4 * NSYM;
    const double det = d00 * m11 - m00 * d11;
    double MC[27], KD[27];
    for (int q = 0; q < 27; ++q) MC[q] = KD[q] = 0.0;
    for (int o = 0; o < 8; ++o) {
        const int ox = o & 1, oy = (o >> 1) & 1, oz = o >> 2;
        const int ex = i - 1 + ox, ey = jj - 1 + oy, ez = kk - 1 + oz;
        if (ex < 0 || ex >= g.nex || ey < 0 || ey >= g.ney || ez < 0 || ez >= g.nez) continue;
        const long long se = ((long long)ez * g.ney + ey) * g.nex + ex;
        const double* A = op.elem + elem_index(op, 1, se) * NV;
        const int as = (~o) & 7;
        for (int bn = 0; bn < 8; ++bn) {
            const double f00 = A[0 * NSYM + symidx<NS>(as, bn)], f11 = A[3 * NSYM + symidx<NS>(as, bn)];
            const int q = ((oz + (bn >> 2)) * 3 + oy + ((bn >> 1) & 1)) * 3 + ox + (bn & 1);
            MC[q] += (f00 * m11 - f11 * m00) / det;
            KD[q] += (d00 * f11 - d11 * f00) / det;
        }
    }
    for (int q = 0; q < 27; ++q) {
        out[q * P + p] = (float)MC[q];
        out[(27 + q) * P + p] = (float)KD[q];
    }
}

void launch_x3_stencil(const OpLc<double>& op, const double Dt[4], const double Mt[4], float* out, cudaStream_t s) {
    const long long P = op.g.plane;
    k_x3_stencil<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(op, Dt[0], Dt[3], Mt[0], Mt[3], out);
}

}  // namespace st
