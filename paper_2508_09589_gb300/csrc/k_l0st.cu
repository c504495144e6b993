// Level-0 operator rows for space-time designs in two space dimensions (FP32 multigrid), as
// time-marching kernels.  The fine operator is matrix free: row n at spatial node p is the sum
// over the four spatial elements e around p and the slabs below (n - 1) and above (n) of
//   C_e (D_t (x) M_x) + k_e (M_t (x) K_x)      (Sec. 2.2, element factorisation)
// with D_t = [[0, 0], [-1, 1]] (upwind in time), M_t = dt/6 [[2, 1], [1, 2]] and C_e, k_e the
// SIMP laws of the element's design value in that slab.  With the node at corner a of element
// e and SM_e(q) = sum_b M_x[a^b] x_q(b), SK_e(q) = sum_b K_x[a^b] x_q(b) over the element's
// four nodes on plane q, plane q adds to the rows it touches (c^s = C_e, d^s = dt/6 k_e of
// slab s):
//   A:   row q + 1: -c^q SM + d^q SK,       row q: c^{q-1} SM + 2 (d^{q-1} + d^q) SK,   row q - 1: d^{q-1} SK
//   A^T: row q + 1:  d^q SK,                row q: (the same),                          row q - 1: -c^{q-1} SM + d^{q-1} SK
// Prescribed neighbours (the t = 0 plane and the spatial Dirichlet set) contribute nothing;
// prescribed rows are the identity.
//
// A block owns a 32 x 8 tile of spatial nodes and a chunk of time planes.  Per plane, the
// halo rows (34 x 10 cells) of the input vectors are staged by cp.async as the 16-byte chunks
// that cover them (a row sits at a per-row offset inside its first chunk) into a ring PF planes
// ahead, with the BF16 design of the slab above (33 x 9 elements; the design buffer carries 8
// values of padding, so every chunk that starts inside it is copied whole).  One pass forms x (u D^-1 in
// the smoother, masked at prescribed cells) in place; another converts the slab's design to
// (C, dt/6 k) per element once; each thread then reads its 3 x 3 neighbourhood and the four
// elements' coefficients and adds the three row parts.  Modes:
//   0: w = A D^-1 u (smoother apply; prescribed rows: u d)
//   1: r = b - A x (residual; prescribed rows: b - x)
//   2: u_0 = b - A x and ||u_0||^2 (smoother start on a nonzero iterate)
//   3: y = A x (operator apply; prescribed rows: x)
#include <mutex>

#include "k_ring.cuh"

namespace st {

namespace {

struct L0stRing {
    static constexpr int VW = 4;                  // floats per chunk
    static constexpr int ROWC = 10, ROW = 40;     // chunks / staged floats per halo row (34 cells, any offset)
    static constexpr int PLANE = 10 * ROW;        // one vector-plane of the tile
    static constexpr int NCH = 10 * ROWC;         // chunk positions per vector-plane
    static constexpr int GW = 8;                  // BF16 per chunk
    static constexpr int GROWC = 5, GROW = 40;    // chunks / staged BF16 per element row (33 elements)
    static constexpr int GCH = 9 * GROWC;         // chunk positions per slab (9 element rows)
    static constexpr int NE = 33 * 9;             // elements per slab that touch the tile
    static constexpr int PF = 8;                  // planes issued ahead
    static constexpr int RING = PF + 1;           // plus the plane whose stencil is being applied
    static constexpr int NPAIR = PLANE / 2;       // x-forming units
};

template <int NQ>
struct L0stLayout {
    using R = L0stRing;
    static constexpr unsigned PLANEB = R::PLANE * 4;
    static constexpr unsigned GSLABB = 9 * R::GROW * 2;
    static constexpr unsigned SLOTB = NQ * PLANEB + GSLABB;  // a multiple of 16
    static constexpr unsigned CKB = R::NE * 8;               // (C, dt/6 k) per element of one slab
    static constexpr unsigned CK0 = R::RING * SLOTB;         // three converted slabs after the ring
    static constexpr size_t smem = (size_t)CK0 + 3 * CKB;
    static_assert(SLOTB % 16 == 0, "slots start on 16-byte boundaries");
};

}  // namespace

template <int MODE, bool TR>
__global__ void __launch_bounds__(256) km_l0st(OpL0<float> op, int chunk, const float* __restrict__ u,
                                               const float* __restrict__ dinv, const float* __restrict__ b,
                                               float* __restrict__ out, int j, int steps, SmState* st_, RedBuf rb) {
    pdl_enter();
    using R = L0stRing;
    constexpr int NQ = MODE == 0 ? 2 : 1;  // staged vectors: u and D^-1, or x
    using LY = L0stLayout<NQ>;
    constexpr int ROW = R::ROW, ROWC = R::ROWC, M = R::VW - 1, PF = R::PF, RING = R::RING;
    constexpr unsigned PLANEB = LY::PLANEB, SLOTB = LY::SLOTB, ROWB = ROW * 4;
    if constexpr (MODE == 0) {
        const SmStateT<float>* st = smt<float>(st_);
        if (st->stop || j >= st->kdim) return;
    }
    const Geom& g = op.g;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 8;
    const int i = i0 + tx, jj = j0 + ty;
    const int nt = g.net, nx1 = g.nx1, ny1 = g.ny1, nex = g.nex, ney = g.ney;
    const int n0 = blockIdx.z * chunk;
    const int n1 = min(n0 + chunk, nt + 1);
    const int ms = n0 > 0 ? n0 - 1 : 0;  // planes [ms, me] feed rows [n0, n1)
    const int me = n1 <= nt ? n1 : nt;
    const int P = (int)g.plane;
    const int N = (int)g.nnodes;
    const int SP = (int)g.sp_elems;
    const int NG = nt * SP;  // design values (one per space-time element)
    const bool in = i < nx1 && jj < ny1;
    const int p = in ? jj * nx1 + i : 0;
    const bool dirp = in ? sp_dir<2>(g, i, jj, 0) : true;
    const unsigned cwin = (unsigned)__cvta_generic_to_shared(g_step_smem);

    // copy role: threads < NQ NCH a chunk position of one staged vector, the next GCH threads a
    // chunk position of the slab's design
    const bool cvec = tid < NQ * R::NCH;
    const bool cdes = !cvec && tid < NQ * R::NCH + R::GCH;
    const int cv = cvec ? tid / R::NCH : 0;
    const int cpos = cvec ? tid - cv * R::NCH : (cdes ? tid - NQ * R::NCH : 0);
    const int crowc = cvec ? ROWC : R::GROWC;
    const int ccy = cpos / crowc, cch = cpos - ccy * crowc;
    const int cgy = j0 - 1 + ccy;  // halo node row, or element row
    const bool crow = cvec ? (cgy >= 0 && cgy < ny1) : (cdes && cgy >= 0 && cgy < ney);
    const int crowE = cvec ? cgy * nx1 + (i0 - 1) : cgy * nex + (i0 - 1);
    const unsigned cdst =
        cwin + (cvec ? (unsigned)cv * PLANEB + 4u * (unsigned)(ccy * ROW + cch * R::VW)
                     : NQ * PLANEB + 2u * (unsigned)(ccy * R::GROW + cch * R::GW));
    const float* csrc = cv == 0 ? u : dinv;
    const __nv_bfloat16* gsrc = op.g16;
    // x-forming role: the element pair at ue of halo row uy (threads < NPAIR)
    const bool uthr = tid < R::NPAIR;
    const int uy = uthr ? tid / (ROW / 2) : 0;
    const int ue = uthr ? 2 * (tid - uy * (ROW / 2)) : 0;
    const int urowE = (j0 - 1 + uy) * nx1 + (i0 - 1);
    const unsigned usrc = 4u * (unsigned)(uy * ROW + ue);
    const int uroff = urowE & M;
    // for each row offset s: which of the pair's two cells are prescribed (2 bits)
    unsigned umask = 0;
#pragma unroll
    for (int sh = 0; sh <= M; ++sh)
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const int ci = i0 - 1 + ue + l - sh, cj = j0 - 1 + uy;
            if (ci >= 0 && ci < nx1 && cj >= 0 && cj < ny1 && sp_dir<2>(g, ci, cj, 0)) umask |= 1u << (2 * sh + l);
        }
    // stencil rows ty .. ty + 2 of the halo tile: their offsets on plane 0
    int roff[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) roff[d] = ((j0 - 1 + ty + d) * nx1 + (i0 - 1)) & M;
    const unsigned gbase = 4u * (unsigned)(ty * ROW + tx);
    // the four elements o around the node (element (i - 1 + (o & 1), j - 1 + (o >> 1))) in the
    // converted slab arrays
    const unsigned eoff = 8u * (unsigned)(ty * 33 + tx);
    const float mx0 = op.mxd[0], mx1 = op.mxd[1], mx2 = op.mxd[2], mx3 = op.mxd[3];
    const float kx0 = op.kxd[0], kx1 = op.kxd[1], kx2 = op.kxd[2], kx3 = op.kxd[3];
    const float dt6 = op.dt6;
    const Simp sp = op.simp;
    const float cins = (float)sp.C_ins, cd = (float)sp.dC, kins = (float)sp.k_ins, kd = (float)sp.dk;

    auto issue = [&](int m, int k) {  // plane m (vectors) and slab m (design) into slot k
        if ((cvec || cdes) && m <= me) {
            const unsigned d = cdst + (unsigned)k * SLOTB;
            if (cvec) {
                const int E = m * P + crowE;
                const int A = (E & ~M) + cch * R::VW;
                int bytes = crow ? 16 : 0;
                if (m == 0 || m == nt) {  // the chunk may begin before the vector or run past its end
                    bytes = 0;
                    if (crow && A >= 0 && A < N) bytes = A <= N - R::VW ? 16 : (N - A) * 4;
                }
                cp_async16(d, csrc + (bytes ? A : 0), bytes);
            } else {
                const int E = m * SP + crowE;
                const int A = (E & ~(R::GW - 1)) + cch * R::GW;
                // whole chunks: the design buffer carries 8 values of padding after its end
                const int bytes = (crow && m < nt && A >= 0 && A < NG) ? 16 : 0;
                cp_async16(d, gsrc + (bytes ? A : 0), bytes);
            }
        }
        cp_async_commit();
    };
    // x of plane m in slot k at this thread's pair, in place over the first staged vector
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
    // (C, dt/6 k) of slab s (staged in slot k) into converted array kc; zero where the element
    // does not exist
    auto convert = [&](int s, int k, int kc) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int e = tid + 256 * r;
            if (e < R::NE) {
                const int ly = e / 33, lx = e - ly * 33;
                const int ex = i0 - 1 + lx, ey = j0 - 1 + ly;
                float c = 0.f, dk = 0.f;
                if (s >= 0 && s < nt && ex >= 0 && ex < nex && ey >= 0 && ey < ney) {
                    const int sg = (s * SP + ey * nex + (i0 - 1)) & (R::GW - 1);
                    const unsigned short raw = *reinterpret_cast<const unsigned short*>(
                        g_step_smem + (unsigned)k * SLOTB + NQ * PLANEB + 2u * (unsigned)(ly * R::GROW + sg + lx));
                    const float gm = __bfloat162float(__ushort_as_bfloat16(raw));
                    c = cins + cd * ipow(gm, sp.p_c);
                    dk = dt6 * (kins + kd * ipow(gm, sp.p_k));
                }
                *reinterpret_cast<float2*>(g_step_smem + LY::CK0 + (unsigned)kc * LY::CKB + 8u * (unsigned)e) =
                    make_float2(c, dk);
            }
        }
    };
    float nrm = 0.f;
    // row r complete at the node: emit it (prescribed rows: the identity)
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

    // prologue: the design of slab ms - 1 (group 0), planes ms .. ms + PF - 1 (groups 1 .. PF)
    {
        const bool keep = cvec;  // only the design copies of the slab below
        if (!keep && cdes && ms - 1 >= 0) {
            const int s = ms - 1;
            const unsigned d = cdst + (unsigned)(RING - 1) * SLOTB;
            const int E = s * SP + crowE;
            const int A = (E & ~(R::GW - 1)) + cch * R::GW;
            const int bytes = (crow && A >= 0 && A < NG) ? 16 : 0;
            cp_async16(d, gsrc + (bytes ? A : 0), bytes);
        }
        cp_async_commit();
    }
#pragma unroll 1
    for (int d = 0; d < PF; ++d) issue(ms + d, d);
    cp_async_wait<PF - 1>();  // slab ms - 1 and plane ms
    __syncthreads();
    convert(ms - 1, RING - 1, 0);
    convert(ms, 0, 1);
    form_x(ms, 0);
    // converted slabs rotate through three arrays: slab s in (s - ms + 1) mod 3
    float cP[4], dP[4];  // slab m - 1 of the node's four elements
    float aP = 0.f, aC = 0.f;  // rows m - 1 and m
    int km = 0, kc = 1;   // ring slot of plane m, converted array of slab m
    bool first = true;
#pragma unroll 1
    for (int m = ms; m <= me; ++m) {
        cp_async_wait<PF - 2>();  // plane m + 1
        __syncthreads();
        const int k1 = km + 1 == RING ? 0 : km + 1;
        const int kc1 = kc == 2 ? 0 : kc + 1;
        const int kcp = kc == 0 ? 2 : kc - 1;
        issue(m + PF, km == 0 ? RING - 1 : km - 1);  // into the slot of plane m - 1
        if (m + 1 <= me) {
            form_x(m + 1, k1);
            convert(m + 1, k1, kc1);
        }
        if (first) {  // slab m - 1 from its converted array
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const float2 v = *reinterpret_cast<const float2*>(
                    g_step_smem + LY::CK0 + (unsigned)kcp * LY::CKB + eoff + 8u * (unsigned)((o >> 1) * 33 + (o & 1)));
                cP[o] = v.x;
                dP[o] = v.y;
            }
            first = false;
        }
        // the node's 3 x 3 neighbourhood of x on plane m
        const int mp = (m * P) & M;
        const unsigned base = gbase + (unsigned)km * SLOTB;
        const unsigned r0 = base + 4u * (unsigned)((mp + roff[0]) & M);
        const unsigned r1 = base + ROWB + 4u * (unsigned)((mp + roff[1]) & M);
        const unsigned r2 = base + 2 * ROWB + 4u * (unsigned)((mp + roff[2]) & M);
        float v[9];
        v[0] = lds1<float>(r0), v[1] = lds1<float>(r0 + 4), v[2] = lds1<float>(r0 + 8);
        v[3] = lds1<float>(r1), v[4] = lds1<float>(r1 + 4), v[5] = lds1<float>(r1 + 8);
        v[6] = lds1<float>(r2), v[7] = lds1<float>(r2 + 4), v[8] = lds1<float>(r2 + 8);
        float aN = 0.f;  // row m + 1
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            const float2 cc = *reinterpret_cast<const float2*>(
                g_step_smem + LY::CK0 + (unsigned)kc * LY::CKB + eoff + 8u * (unsigned)((o >> 1) * 33 + (o & 1)));
            const int ox = o & 1, oy = o >> 1;
            const int as = (~o) & 3;  // the node's corner in element o
            // the element's nodes bs = (bx, by): neighbourhood cell (oy + by) * 3 + ox + bx
            const float x00 = v[oy * 3 + ox], x10 = v[oy * 3 + ox + 1], x01 = v[(oy + 1) * 3 + ox],
                        x11 = v[(oy + 1) * 3 + ox + 1];
            // M_x[a ^ b] and K_x[a ^ b] for the corner a = as and the four nodes b
            const float m00 = as == 0 ? mx0 : as == 1 ? mx1 : as == 2 ? mx2 : mx3;  // b = 0
            const float m10 = as == 1 ? mx0 : as == 0 ? mx1 : as == 3 ? mx2 : mx3;  // b = 1
            const float m01 = as == 2 ? mx0 : as == 3 ? mx1 : as == 0 ? mx2 : mx3;  // b = 2
            const float m11 = as == 3 ? mx0 : as == 2 ? mx1 : as == 1 ? mx2 : mx3;  // b = 3
            const float k00 = as == 0 ? kx0 : as == 1 ? kx1 : as == 2 ? kx2 : kx3;
            const float k10 = as == 1 ? kx0 : as == 0 ? kx1 : as == 3 ? kx2 : kx3;
            const float k01 = as == 2 ? kx0 : as == 3 ? kx1 : as == 0 ? kx2 : kx3;
            const float k11 = as == 3 ? kx0 : as == 2 ? kx1 : as == 1 ? kx2 : kx3;
            const float SM = m00 * x00 + m10 * x10 + m01 * x01 + m11 * x11;
            const float SK = k00 * x00 + k10 * x10 + k01 * x01 + k11 * x11;
            const float cq = cc.x, dq = cc.y, cq1 = cP[o], dq1 = dP[o];
            if constexpr (!TR) {
                aN += dq * SK - cq * SM;
                aP += dq1 * SK;
            } else {
                aN += dq * SK;
                aP += dq1 * SK - cq1 * SM;
            }
            aC += cq1 * SM + 2.f * (dq1 + dq) * SK;
            cP[o] = cq;
            dP[o] = dq;
        }
        if (in && m - 1 >= n0 && m - 1 < n1) emit(m - 1, aP);
        if (in && m == nt && nt >= n0 && nt < n1) emit(nt, aC);
        aP = aC;
        aC = aN;
        km = k1;
        kc = kc1;
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
void launch_l0st_t(const OpL0<float>& op, const float* u, const float* dinv, const float* b, float* out, int j,
                   int steps, SmState* st, RedBuf rb, cudaStream_t s) {
    dim3 grid, block;
    const MarchGrid mg = march_grid(op.g, grid, block);
    constexpr size_t bytes = L0stLayout<MODE == 0 ? 2 : 1>::smem;
    static std::once_flag attr;
    std::call_once(attr, [] {
        cudaFuncSetAttribute(km_l0st<MODE, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    });
    launch_pdl(km_l0st<MODE, TR>, grid, block, bytes, s, op, mg.chunk, u, dinv, b, out, j, steps, st, rb);
}
}  // namespace

bool l0st_usable(const OpL0<float>& op, const void* const* vecs, int nvec) {
    if (op.tc || op.g.nz1 != 1 || op.g16 == nullptr) return false;  // space-time 2-D designs only
    if (op.g.nnodes > (1LL << 31) - 64 || (long long)op.g.net * op.g.sp_elems > (1LL << 31) - 64) return false;
    if (op.g.plane < 64) return false;  // the chunks of a plane's last halo row end inside the next plane
    auto ok = [](const void* q) { return ((uintptr_t)q & 15u) == 0; };
    if (!ok(op.g16)) return false;
    for (int q = 0; q < nvec; ++q)
        if (vecs[q] && !ok(vecs[q])) return false;
    return true;
}

void launch_l0st(int mode, bool tr, const OpL0<float>& op, const float* u, const float* dinv, const float* b,
                 float* out, int j, int steps, SmState* st, RedBuf rb, cudaStream_t s) {
    if (mode == 0)
        tr ? launch_l0st_t<0, true>(op, u, dinv, b, out, j, steps, st, rb, s)
           : launch_l0st_t<0, false>(op, u, dinv, b, out, j, steps, st, rb, s);
    else if (mode == 1)
        tr ? launch_l0st_t<1, true>(op, u, dinv, b, out, j, steps, st, rb, s)
           : launch_l0st_t<1, false>(op, u, dinv, b, out, j, steps, st, rb, s);
    else if (mode == 2)
        tr ? launch_l0st_t<2, true>(op, u, dinv, b, out, j, steps, st, rb, s)
           : launch_l0st_t<2, false>(op, u, dinv, b, out, j, steps, st, rb, s);
    else
        tr ? launch_l0st_t<3, true>(op, u, dinv, b, out, j, steps, st, rb, s)
           : launch_l0st_t<3, false>(op, u, dinv, b, out, j, steps, st, rb, s);
}

}  // namespace st
