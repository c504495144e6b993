// Level-0 operator rows for extruded (time-constant) designs in three space dimensions (FP32
// multigrid), as time-marching kernels.  With the design constant in time, every element has
// the same C_e and k_e in each slab, so the element sums of Sec. 2.2's factorisation
// C_e (D_t (x) M_x) + k_e (M_t (x) K_x) collapse, per node, to two time-constant 27-point
// spatial stencils: MC = sum_e C_e M_x (the node's row of the C-weighted mass matrix) and
// KD = sum_e dt/6 k_e K_x.  With sM = MC x_q and sK = KD x_q on plane q and e_s = 1 when slab
// s exists (0 <= s < n_t), plane q adds to the rows it touches:
//   A:   row q + 1: e_q (sK - sM),   row q: e_{q-1} sM + 2 (e_{q-1} + e_q) sK,   row q - 1: e_{q-1} sK
//   A^T: row q + 1: e_q sK,          row q: (the same),                          row q - 1: e_{q-1} (sK - sM)
// Prescribed neighbours (the t = 0 plane and the spatial Dirichlet set) contribute nothing;
// prescribed rows are the identity.
//
// A block owns a 16 x 4 x 4 tile of spatial nodes and a chunk of time planes; each thread
// builds its node's two stencils once from the BF16 design of the eight elements around it.
// Per plane, the 36 halo rows (18 x 6 x 6 cells) of the input vectors are staged by cp.async
// as the 16-byte chunks that cover them into a ring PF planes ahead; one pass forms x (u D^-1
// in the smoother, masked at prescribed cells) into a double-buffered plane at fixed
// positions; each thread reads its 27 neighbours from it.  Modes as in k_l0st.cu:
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

template <int MODE, bool TR>
__global__ void __launch_bounds__(256, 2) km_l0x3(OpL0<float> op, int chunk, int gyt, const float* __restrict__ u,
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

    // the node's two stencils from the eight elements around it (BF16 design, constant in time)
    float MC[27], KD[27];
#pragma unroll
    for (int q = 0; q < 27; ++q) MC[q] = KD[q] = 0.f;
    if (in) {
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
        float aN;
        if constexpr (!TR) {
            aN = eq * (sK - sM);
            aP += eq1 * sK;
        } else {
            aN = eq * sK;
            aP += eq1 * (sK - sM);
        }
        aC += eq1 * sM + 2.f * (eq1 + eq) * sK;
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
template <int MODE, bool TR>
void launch_l0x3_t(const OpL0<float>& op, const float* u, const float* dinv, const float* b, float* out, int j,
                   int steps, SmState* st, RedBuf rb, cudaStream_t s) {
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
        cudaFuncSetAttribute(km_l0x3<MODE, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    });
    launch_pdl(km_l0x3<MODE, TR>, dim3((unsigned)gx, (unsigned)(gyt * gzt), (unsigned)gz), dim3(256), bytes, s, op,
               chunk, gyt, u, dinv, b, out, j, steps, st, rb);
}
}  // namespace

bool l0x3_usable(const OpL0<float>& op, const void* const* vecs, int nvec) {
    if (!op.tc || op.g.nz1 <= 1 || op.g16 == nullptr) return false;  // extruded 3-D designs only
    if (op.g.nnodes > (1LL << 31) - 64) return false;
    if (op.g.plane < 64) return false;  // the chunks of a plane's last halo row end inside the next plane
    const long long gyz = (long long)((op.g.ny1 + 3) / 4) * ((op.g.nz1 + 3) / 4);
    if (gyz > 65535) return false;  // grid.y
    auto ok = [](const void* q) { return ((uintptr_t)q & 15u) == 0; };
    for (int q = 0; q < nvec; ++q)
        if (vecs[q] && !ok(vecs[q])) return false;
    return true;
}

void launch_l0x3(int mode, bool tr, const OpL0<float>& op, const float* u, const float* dinv, const float* b,
                 float* out, int j, int steps, SmState* st, RedBuf rb, cudaStream_t s) {
    if (mode == 0)
        tr ? launch_l0x3_t<0, true>(op, u, dinv, b, out, j, steps, st, rb, s)
           : launch_l0x3_t<0, false>(op, u, dinv, b, out, j, steps, st, rb, s);
    else if (mode == 1)
        tr ? launch_l0x3_t<1, true>(op, u, dinv, b, out, j, steps, st, rb, s)
           : launch_l0x3_t<1, false>(op, u, dinv, b, out, j, steps, st, rb, s);
    else if (mode == 2)
        tr ? launch_l0x3_t<2, true>(op, u, dinv, b, out, j, steps, st, rb, s)
           : launch_l0x3_t<2, false>(op, u, dinv, b, out, j, steps, st, rb, s);
    else
        tr ? launch_l0x3_t<3, true>(op, u, dinv, b, out, j, steps, st, rb, s)
           : launch_l0x3_t<3, false>(op, u, dinv, b, out, j, steps, st, rb, s);
}

}  // namespace st
