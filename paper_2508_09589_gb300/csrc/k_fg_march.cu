// FP64 level-0 operator rows of the outer FGMRES (Sec. 3.2) for space-time 2-D designs and
// extruded 3-D designs, as time-marching kernels (the same row formulas as the FP32 marching
// kernels of k_l0st.cu and k_l0x3.cu, in FP64 from the FP64 design).  Modes:
//   0: w = J z (z in the preconditioner's precision TZ; prescribed rows: z), and z copied into
//      the Krylov basis when zstore is given (the FGMRES apply; with TZ = double and no zstore,
//      the plain FP64 apply)
//   1: r = f - J x and ||r||^2 into the FGMRES state (the residual of a restart cycle)
// 2-D (km_fgst): per plane the FP64 design of the slab above the 32 x 8 tile (33 x 9 elements)
// is staged with z and converted once to (C, dt/6 k); each node adds its four elements' mass and
// stiffness products to rows m + 1, m and m - 1.  3-D (km_fgx3): each thread holds its node's
// two FP64 27-point stencils (C-weighted mass, dt/6 k-weighted stiffness) for the whole march.
// The input is staged by 16-byte cp.async chunks into a ring PF planes ahead and x (masked at
// prescribed cells, in FP64) is formed into a double-buffered plane.  FP64 FMA throughput bounds
// both on this GPU.
#include <mutex>

#include "k_ring.cuh"

namespace st {

namespace {

template <typename TZ>
struct FgstRing {
    static constexpr int VW = 16 / (int)sizeof(TZ);                 // input values per chunk
    static constexpr int ROWC = (VW - 1 + 34 + VW - 1) / VW, ROW = ROWC * VW;
    static constexpr int PLANE = 10 * ROW, NCH = 10 * ROWC;
    static constexpr int GROWC = 18, GROW = 36;                     // FP64 design: chunks / values per element row
    static constexpr int GCH = 9 * GROWC;
    static constexpr int NE = 33 * 9;
    static constexpr int PF = 8, RING = PF + 1;
    static constexpr unsigned PLANEB = PLANE * sizeof(TZ);
    static constexpr unsigned GSLABB = 9 * GROW * 8;
    static constexpr unsigned SLOTB = PLANEB + GSLABB;
    static constexpr unsigned XB0 = RING * SLOTB;                   // two FP64 x planes (staged layout)
    static constexpr unsigned XPB = PLANE * 8;
    static constexpr unsigned CK0 = XB0 + 2 * XPB;                  // three converted slabs (C, dt/6 k)
    static constexpr unsigned CKB = NE * 16;
    static constexpr size_t smem = (size_t)CK0 + 3 * CKB;
    static constexpr int UNITS = (NCH + GCH + 255) / 256;          // copy units per thread
    static_assert(SLOTB % 16 == 0 && XB0 % 16 == 0 && CK0 % 16 == 0, "16-byte aligned regions");
};

template <typename TZ>
struct Fgx3Ring {
    static constexpr int TX = 16, TY = 4, TZN = 4, HX = 18, HY = 6, HZ = 6, NROW = HY * HZ;
    static constexpr int VW = 16 / (int)sizeof(TZ);
    static constexpr int ROWC = (VW - 1 + HX + VW - 1) / VW, ROW = ROWC * VW;
    static constexpr int PLANE = NROW * ROW, NCH = NROW * ROWC, NX = NROW * HX;
    static constexpr int PF = 8, RING = PF;
    static constexpr unsigned SLOTB = PLANE * sizeof(TZ);
    static constexpr unsigned XB0 = RING * SLOTB, XPB = NX * 8;
    static constexpr size_t smem = (size_t)XB0 + 2 * XPB;
    static constexpr int UNITS = (NCH + 255) / 256, XUNITS = (NX + 255) / 256;
    static_assert(SLOTB % 16 == 0 && XB0 % 16 == 0, "16-byte aligned regions");
};

}  // namespace

// ---------------------------------------------------------------- 2-D space-time designs
template <int MODE, bool TR, typename TZ>
__global__ void __launch_bounds__(256) km_fgst(OpL0<double> op, int chunk, const TZ* __restrict__ z,
                                               TZ* __restrict__ zstore, const double* __restrict__ f,
                                               double* __restrict__ out, FgState* fs, RedBuf rb) {
    pdl_enter();
    using R = FgstRing<TZ>;
    constexpr int ROW = R::ROW, ROWC = R::ROWC, M = R::VW - 1, PF = R::PF, RING = R::RING;
    constexpr unsigned ES = sizeof(TZ), SLOTB = R::SLOTB, ROWB8 = ROW * 8;
    const Geom& g = op.g;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 8;
    const int i = i0 + tx, jj = j0 + ty;
    const int nt = g.net, nx1 = g.nx1, ny1 = g.ny1, nex = g.nex, ney = g.ney;
    const int n0 = blockIdx.z * chunk;
    const int n1 = min(n0 + chunk, nt + 1);
    const int ms = n0 > 0 ? n0 - 1 : 0;
    const int me = n1 <= nt ? n1 : nt;
    const int P = (int)g.plane, N = (int)g.nnodes, SP = (int)g.sp_elems, NG = nt * SP;
    const bool in = i < nx1 && jj < ny1;
    const int p = in ? jj * nx1 + i : 0;
    const bool dirp = in ? sp_dir<2>(g, i, jj, 0) : true;
    const unsigned cwin = (unsigned)__cvta_generic_to_shared(g_step_smem);

    // copy units c = tid + 256 r: input chunk positions, then design chunk positions
    int cE[R::UNITS], cch[R::UNITS], ckind[R::UNITS];  // kind 0 none, 1 input, 2 design
    bool crow[R::UNITS];
    unsigned cdst[R::UNITS];
#pragma unroll
    for (int r = 0; r < R::UNITS; ++r) {
        const int c = tid + 256 * r;
        ckind[r] = c < R::NCH ? 1 : (c < R::NCH + R::GCH ? 2 : 0);
        const int pos = ckind[r] == 1 ? c : (ckind[r] == 2 ? c - R::NCH : 0);
        const int rc = ckind[r] == 1 ? ROWC : R::GROWC;
        const int cy = pos / rc;
        cch[r] = pos - cy * rc;
        const int gy = j0 - 1 + cy;
        crow[r] = ckind[r] == 1 ? (gy >= 0 && gy < ny1) : (ckind[r] == 2 && gy >= 0 && gy < ney);
        cE[r] = ckind[r] == 1 ? gy * nx1 + (i0 - 1) : gy * nex + (i0 - 1);
        cdst[r] = cwin + (ckind[r] == 1 ? ES * (unsigned)(cy * ROW + cch[r] * R::VW)
                                        : R::PLANEB + 8u * (unsigned)(cy * R::GROW + cch[r] * 2));
    }
    // x-forming pairs (staged positions ue, ue + 1 of halo row uy)
    const bool uthr = tid < R::PLANE / 2;
    const int uy = uthr ? tid / (ROW / 2) : 0;
    const int ue = uthr ? 2 * (tid - uy * (ROW / 2)) : 0;
    const int uroff = ((j0 - 1 + uy) * nx1 + (i0 - 1)) & M;
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
    const unsigned gbase = 8u * (unsigned)(ty * ROW + tx);
    const unsigned eoff = 16u * (unsigned)(ty * 33 + tx);
    const double mx0 = op.mxd[0], mx1 = op.mxd[1], mx2 = op.mxd[2], mx3 = op.mxd[3];
    const double kx0 = op.kxd[0], kx1 = op.kxd[1], kx2 = op.kxd[2], kx3 = op.kxd[3];
    const double dt6 = op.dt6;
    const Simp sp = op.simp;

    auto issue = [&](int m, int k) {
        if (m <= me) {
#pragma unroll
            for (int r = 0; r < R::UNITS; ++r) {
                if (ckind[r] == 1) {
                    const int E = m * P + cE[r];
                    const int A = (E & ~M) + cch[r] * R::VW;
                    int bytes = crow[r] ? 16 : 0;
                    if (m == 0 || m == nt) {
                        bytes = 0;
                        if (crow[r] && A >= 0 && A < N) bytes = A <= N - R::VW ? 16 : (N - A) * (int)ES;
                    }
                    cp_async16(cdst[r] + (unsigned)k * SLOTB, z + (bytes ? A : 0), bytes);
                } else if (ckind[r] == 2) {
                    // whole chunks: the FP64 design buffer carries padding after its end
                    const int E = m * SP + cE[r];
                    const int A = (E & ~1) + cch[r] * 2;
                    const int bytes = (crow[r] && m < nt && A >= 0 && A < NG) ? 16 : 0;
                    cp_async16(cdst[r] + (unsigned)k * SLOTB, op.g64 + (bytes ? A : 0), bytes);
                }
            }
        }
        cp_async_commit();
    };
    auto form_x = [&](int m, int k, int xb) {
        if (!uthr) return;
        const unsigned a = (unsigned)k * SLOTB + ES * (unsigned)(uy * ROW + ue);
        TZ z0, z1;
        lds2<TZ>(a, z0, z1);
        double x0 = (double)z0, x1 = (double)z1;
        const unsigned o = m == 0 ? 3u : (umask >> (2 * ((m * P + uroff) & M))) & 3u;
        if (o & 1u) x0 = 0.0;
        if (o & 2u) x1 = 0.0;
        sts2<double>(R::XB0 + (unsigned)xb * R::XPB + 8u * (unsigned)(uy * ROW + ue), x0, x1);
    };
    auto convert = [&](int s, int k, int kc) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int e = tid + 256 * r;
            if (e < R::NE) {
                const int ly = e / 33, lx = e - ly * 33;
                const int ex = i0 - 1 + lx, ey = j0 - 1 + ly;
                double c = 0.0, dk = 0.0;
                if (s >= 0 && s < nt && ex >= 0 && ex < nex && ey >= 0 && ey < ney) {
                    const int sg = (s * SP + ey * nex + (i0 - 1)) & 1;
                    const double gm =
                        lds1<double>((unsigned)k * SLOTB + R::PLANEB + 8u * (unsigned)(ly * R::GROW + sg + lx));
                    c = sp.C_ins + sp.dC * ipow(gm, sp.p_c);
                    dk = dt6 * (sp.k_ins + sp.dk * ipow(gm, sp.p_k));
                }
                sts2<double>(R::CK0 + (unsigned)kc * R::CKB + 16u * (unsigned)e, c, dk);
            }
        }
    };
    double nrm = 0.0;
    auto emit = [&](int r, double a) {
        const int qn = r * P + p;
        const TZ zq = z[qn];
        const double v = (r == 0 || dirp) ? (double)zq : a;
        if constexpr (MODE == 0) {
            out[qn] = v;
            if (zstore) zstore[qn] = zq;
        } else {
            const double rr = f[qn] - v;
            out[qn] = rr;
            nrm += rr * rr;
        }
    };

    {  // prologue: the design of slab ms - 1 (group 0), planes ms .. ms + PF - 1
#pragma unroll
        for (int r = 0; r < R::UNITS; ++r)
            if (ckind[r] == 2 && ms - 1 >= 0) {
                const int E = (ms - 1) * SP + cE[r];
                const int A = (E & ~1) + cch[r] * 2;
                const int bytes = (crow[r] && A >= 0 && A < NG) ? 16 : 0;
                cp_async16(cdst[r] + (unsigned)(RING - 1) * SLOTB, op.g64 + (bytes ? A : 0), bytes);
            }
        cp_async_commit();
    }
#pragma unroll 1
    for (int d = 0; d < PF; ++d) issue(ms + d, d);
    cp_async_wait<PF - 1>();
    __syncthreads();
    convert(ms - 1, RING - 1, 0);
    convert(ms, 0, 1);
    form_x(ms, 0, ms & 1);
    double cP[4], dP[4];
    double aP = 0.0, aC = 0.0;
    int km = 0, kc = 1;
    bool first = true;
#pragma unroll 1
    for (int m = ms; m <= me; ++m) {
        cp_async_wait<PF - 2>();
        __syncthreads();
        const int k1 = km + 1 == RING ? 0 : km + 1;
        const int kc1 = kc == 2 ? 0 : kc + 1;
        const int kcp = kc == 0 ? 2 : kc - 1;
        issue(m + PF, km == 0 ? RING - 1 : km - 1);
        if (m + 1 <= me) {
            form_x(m + 1, k1, (m + 1) & 1);
            convert(m + 1, k1, kc1);
        }
        if (first) {
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                lds2<double>(R::CK0 + (unsigned)kcp * R::CKB + eoff + 16u * (unsigned)((o >> 1) * 33 + (o & 1)), cP[o],
                             dP[o]);
            }
            first = false;
        }
        const int mp = (m * P) & M;
        const unsigned base = R::XB0 + (unsigned)(m & 1) * R::XPB + gbase;
        const unsigned r0 = base + 8u * (unsigned)((mp + roff[0]) & M);
        const unsigned r1 = base + ROWB8 + 8u * (unsigned)((mp + roff[1]) & M);
        const unsigned r2 = base + 2 * ROWB8 + 8u * (unsigned)((mp + roff[2]) & M);
        double v[9];
        v[0] = lds1<double>(r0), v[1] = lds1<double>(r0 + 8), v[2] = lds1<double>(r0 + 16);
        v[3] = lds1<double>(r1), v[4] = lds1<double>(r1 + 8), v[5] = lds1<double>(r1 + 16);
        v[6] = lds1<double>(r2), v[7] = lds1<double>(r2 + 8), v[8] = lds1<double>(r2 + 16);
        double aN = 0.0;
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            double cq, dq;
            lds2<double>(R::CK0 + (unsigned)kc * R::CKB + eoff + 16u * (unsigned)((o >> 1) * 33 + (o & 1)), cq, dq);
            const int ox = o & 1, oy = o >> 1, as = (~o) & 3;
            const double x00 = v[oy * 3 + ox], x10 = v[oy * 3 + ox + 1], x01 = v[(oy + 1) * 3 + ox],
                         x11 = v[(oy + 1) * 3 + ox + 1];
            const double m00 = as == 0 ? mx0 : as == 1 ? mx1 : as == 2 ? mx2 : mx3;
            const double m10 = as == 1 ? mx0 : as == 0 ? mx1 : as == 3 ? mx2 : mx3;
            const double m01 = as == 2 ? mx0 : as == 3 ? mx1 : as == 0 ? mx2 : mx3;
            const double m11 = as == 3 ? mx0 : as == 2 ? mx1 : as == 1 ? mx2 : mx3;
            const double k00 = as == 0 ? kx0 : as == 1 ? kx1 : as == 2 ? kx2 : kx3;
            const double k10 = as == 1 ? kx0 : as == 0 ? kx1 : as == 3 ? kx2 : kx3;
            const double k01 = as == 2 ? kx0 : as == 3 ? kx1 : as == 0 ? kx2 : kx3;
            const double k11 = as == 3 ? kx0 : as == 2 ? kx1 : as == 1 ? kx2 : kx3;
            const double SM = m00 * x00 + m10 * x10 + m01 * x01 + m11 * x11;
            const double SK = k00 * x00 + k10 * x10 + k01 * x01 + k11 * x11;
            if constexpr (!TR) {
                aN += dq * SK - cq * SM;
                aP += dP[o] * SK;
            } else {
                aN += dq * SK;
                aP += dP[o] * SK - cP[o] * SM;
            }
            aC += cP[o] * SM + 2.0 * (dP[o] + dq) * SK;
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
    if constexpr (MODE == 1) {
        double acc[1] = {nrm};
        __shared__ double red_out[1];
        if (reduce_publish<1>(acc, 1, rb, red_out)) {
            if (tid == 0) fg_residual_finish(fs, red_out[0]);
        }
    }
}

// ---------------------------------------------------------------- 3-D extruded designs
template <int MODE, bool TR, typename TZ>
__global__ void __launch_bounds__(256, 1) km_fgx3(OpL0<double> op, int chunk, int gyt, const TZ* __restrict__ z,
                                                  TZ* __restrict__ zstore, const double* __restrict__ f,
                                                  double* __restrict__ out, FgState* fs, RedBuf rb) {
    pdl_enter();
    using R = Fgx3Ring<TZ>;
    constexpr int M = R::VW - 1, PF = R::PF, RING = R::RING;
    constexpr unsigned ES = sizeof(TZ), SLOTB = R::SLOTB;
    const Geom& g = op.g;
    const int t = threadIdx.x;
    const int tx = t & 15, ty = (t >> 4) & 3, tz = t >> 6;
    const int i0 = blockIdx.x * R::TX, j0 = (blockIdx.y % gyt) * R::TY, k0 = (blockIdx.y / gyt) * R::TZN;
    const int i = i0 + tx, jj = j0 + ty, kk = k0 + tz;
    const int nt = g.net, nx1 = g.nx1, ny1 = g.ny1, nz1 = g.nz1;
    const int n0 = blockIdx.z * chunk;
    const int n1 = min(n0 + chunk, nt + 1);
    const int ms = n0 > 0 ? n0 - 1 : 0;
    const int me = n1 <= nt ? n1 : nt;
    const int P = (int)g.plane, N = (int)g.nnodes;
    const bool in = i < nx1 && jj < ny1 && kk < nz1;
    const int p = in ? (kk * ny1 + jj) * nx1 + i : 0;
    const bool dirp = in ? sp_dir<3>(g, i, jj, kk) : true;
    const unsigned cwin = (unsigned)__cvta_generic_to_shared(g_step_smem);

    double MC[27], KD[27];
#pragma unroll
    for (int q = 0; q < 27; ++q) MC[q] = KD[q] = 0.0;
    if (in) {
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            const int ox = o & 1, oy = (o >> 1) & 1, oz = o >> 2;
            const int ex = i - 1 + ox, ey = jj - 1 + oy, ez = kk - 1 + oz;
            if (ex < 0 || ex >= g.nex || ey < 0 || ey >= g.ney || ez < 0 || ez >= g.nez) continue;
            const double gm = op.g64[(ez * g.ney + ey) * g.nex + ex];
            const double c = op.simp.C_ins + op.simp.dC * ipow(gm, op.simp.p_c);
            const double dk = op.dt6 * (op.simp.k_ins + op.simp.dk * ipow(gm, op.simp.p_k));
            const int as = (~o) & 7;
#pragma unroll
            for (int bn = 0; bn < 8; ++bn) {
                const int q = ((oz + (bn >> 2)) * 3 + oy + ((bn >> 1) & 1)) * 3 + ox + (bn & 1);
                MC[q] += c * op.mxd[as ^ bn];
                KD[q] += dk * op.kxd[as ^ bn];
            }
        }
    }
    int cE[R::UNITS], cch[R::UNITS];
    unsigned cdst[R::UNITS];
    bool cok[R::UNITS], crow[R::UNITS];
#pragma unroll
    for (int r = 0; r < R::UNITS; ++r) {
        const int c = t + 256 * r;
        cok[r] = c < R::NCH;
        const int pos = cok[r] ? c : 0;
        const int rr = pos / R::ROWC, ch = pos - rr * R::ROWC;
        const int ry = rr % R::HY, rz = rr / R::HY;
        const int gj = j0 - 1 + ry, gk = k0 - 1 + rz;
        crow[r] = cok[r] && gj >= 0 && gj < ny1 && gk >= 0 && gk < nz1;
        cE[r] = (gk * ny1 + gj) * nx1 + (i0 - 1);
        cch[r] = ch;
        cdst[r] = cwin + ES * (unsigned)(rr * R::ROW + ch * R::VW);
    }
    int xsrc[R::XUNITS], xroff[R::XUNITS];
    unsigned xmask[R::XUNITS];
    bool xok[R::XUNITS];
#pragma unroll
    for (int r = 0; r < R::XUNITS; ++r) {
        const int c = t + 256 * r;
        xok[r] = c < R::NX;
        const int rr = xok[r] ? c / R::HX : 0, cx = xok[r] ? c - rr * R::HX : 0;
        const int ry = rr % R::HY, rz = rr / R::HY;
        const int gi = i0 - 1 + cx, gj = j0 - 1 + ry, gk = k0 - 1 + rz;
        xroff[r] = ((gk * ny1 + gj) * nx1 + (i0 - 1)) & M;
        xsrc[r] = rr * R::ROW + cx;
        const bool inside = gi >= 0 && gi < nx1 && gj >= 0 && gj < ny1 && gk >= 0 && gk < nz1;
        xmask[r] = (inside && sp_dir<3>(g, gi, gj, gk)) ? 1u : 0u;
    }
    const unsigned gbase = 8u * (unsigned)((tz * R::HY + ty) * R::HX + tx);

    auto issue = [&](int m, int k) {
        if (m <= me) {
#pragma unroll
            for (int r = 0; r < R::UNITS; ++r) {
                if (!cok[r]) continue;
                const int E = m * P + cE[r];
                const int A = (E & ~M) + cch[r] * R::VW;
                int bytes = crow[r] ? 16 : 0;
                if (m == 0 || m == nt) {
                    bytes = 0;
                    if (crow[r] && A >= 0 && A < N) bytes = A <= N - R::VW ? 16 : (N - A) * (int)ES;
                }
                cp_async16(cdst[r] + (unsigned)k * SLOTB, z + (bytes ? A : 0), bytes);
            }
        }
        cp_async_commit();
    };
    auto form_x = [&](int m, int k, int xb) {
        const int mp = (m * P) & M;
#pragma unroll
        for (int r = 0; r < R::XUNITS; ++r) {
            if (!xok[r]) continue;
            double x = (double)lds1<TZ>((unsigned)k * SLOTB + ES * (unsigned)(xsrc[r] + ((mp + xroff[r]) & M)));
            if (m == 0 || xmask[r]) x = 0.0;
            *reinterpret_cast<double*>(g_step_smem + R::XB0 + (unsigned)xb * R::XPB + 8u * (unsigned)(t + 256 * r)) = x;
        }
    };
    double nrm = 0.0;
    auto emit = [&](int r, double a) {
        const int qn = r * P + p;
        const TZ zq = z[qn];
        const double v = (r == 0 || dirp) ? (double)zq : a;
        if constexpr (MODE == 0) {
            out[qn] = v;
            if (zstore) zstore[qn] = zq;
        } else {
            const double rr = f[qn] - v;
            out[qn] = rr;
            nrm += rr * rr;
        }
    };

#pragma unroll 1
    for (int d = 0; d < PF; ++d) issue(ms + d, d);
    cp_async_wait<PF - 1>();
    __syncthreads();
    form_x(ms, 0, ms & 1);
    double aP = 0.0, aC = 0.0;
    int km = 0;
#pragma unroll 1
    for (int m = ms; m <= me; ++m) {
        cp_async_wait<PF - 2>();
        __syncthreads();
        const int k1 = km + 1 == RING ? 0 : km + 1;
        issue(m + PF, km);
        if (m + 1 <= me) form_x(m + 1, k1, (m + 1) & 1);
        const unsigned xbase = R::XB0 + (unsigned)(m & 1) * R::XPB + gbase;
        double sM = 0.0, sK = 0.0;
#pragma unroll
        for (int dz = 0; dz < 3; ++dz)
#pragma unroll
            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    const int q = (dz * 3 + dy) * 3 + dx;
                    const double v = lds1<double>(xbase + 8u * (unsigned)((dz * R::HY + dy) * R::HX + dx));
                    sM += MC[q] * v;
                    sK += KD[q] * v;
                }
        const double eq = m < nt ? 1.0 : 0.0, eq1 = m >= 1 ? 1.0 : 0.0;
        // level 0: D_t = [[0, 0], [-1, 1]], M_t = [[2, 1], [1, 2]] with dt/6 in KD
        const double aN = eq * (TR ? sK : sK - sM);
        aP += eq1 * (TR ? sK - sM : sK);
        aC += eq1 * (sM + 2.0 * sK) + eq * 2.0 * sK;
        if (in && m - 1 >= n0 && m - 1 < n1) emit(m - 1, aP);
        if (in && m == nt && nt >= n0 && nt < n1) emit(nt, aC);
        aP = aC;
        aC = aN;
        km = k1;
    }
    cp_async_wait<0>();
    if constexpr (MODE == 1) {
        double acc[1] = {nrm};
        __shared__ double red_out[1];
        if (reduce_publish<1>(acc, 1, rb, red_out)) {
            if (t == 0) fg_residual_finish(fs, red_out[0]);
        }
    }
}

// ---------------------------------------------------------------- launchers
namespace {
template <int MODE, bool TR, typename TZ>
void launch_fgst_t(const OpL0<double>& op, const TZ* z, TZ* zstore, const double* f, double* out, FgState* fs,
                   RedBuf rb, cudaStream_t s) {
    dim3 grid, block;
    const MarchGrid mg = march_grid(op.g, grid, block);
    constexpr size_t bytes = FgstRing<TZ>::smem;
    static std::once_flag attr;
    std::call_once(attr, [] {
        cudaFuncSetAttribute(km_fgst<MODE, TR, TZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    });
    launch_pdl(km_fgst<MODE, TR, TZ>, grid, block, bytes, s, op, mg.chunk, z, zstore, f, out, fs, rb);
}

template <int MODE, bool TR, typename TZ>
void launch_fgx3_t(const OpL0<double>& op, const TZ* z, TZ* zstore, const double* f, double* out, FgState* fs,
                   RedBuf rb, cudaStream_t s) {
    using R = Fgx3Ring<TZ>;
    const Geom& g = op.g;
    const int gx = (g.nx1 + R::TX - 1) / R::TX, gyt = (g.ny1 + R::TY - 1) / R::TY, gzt = (g.nz1 + R::TZN - 1) / R::TZN;
    const long long tiles = (long long)gx * gyt * gzt;
    const long long budget = g.march_blocks > 0 && g.march_blocks < kMaxBlocks ? g.march_blocks : kMarchBlocks;
    long long gz = budget / tiles;
    if (gz < 1) gz = 1;
    if (gz > g.nt1) gz = g.nt1;
    const int chunk = (int)((g.nt1 + gz - 1) / gz);
    gz = (g.nt1 + chunk - 1) / chunk;
    constexpr size_t bytes = R::smem;
    static std::once_flag attr;
    std::call_once(attr, [] {
        cudaFuncSetAttribute(km_fgx3<MODE, TR, TZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    });
    launch_pdl(km_fgx3<MODE, TR, TZ>, dim3((unsigned)gx, (unsigned)(gyt * gzt), (unsigned)gz), dim3(256), bytes, s,
               op, chunk, gyt, z, zstore, f, out, fs, rb);
}
}  // namespace

bool fg_march_usable(int sd, const OpL0<double>& op, const void* const* vecs, int nvec) {
    if (!g_l0st || op.g64 == nullptr) return false;
    if (op.g.nnodes > (1LL << 31) - 64 || op.g.plane < 64) return false;
    if (sd == 2) {
        if (op.tc || op.g.nz1 != 1 || op.st_dir) return false;  // space-time 2-D designs
        if ((long long)op.g.net * op.g.sp_elems > (1LL << 31) - 64) return false;
        if (((uintptr_t)op.g64 & 15u) != 0) return false;
    } else {
        if (!op.tc || op.g.nz1 <= 1) return false;  // extruded 3-D designs
        if ((long long)((op.g.ny1 + 3) / 4) * ((op.g.nz1 + 3) / 4) > 65535) return false;
    }
    for (int q = 0; q < nvec; ++q)
        if (vecs[q] && ((uintptr_t)vecs[q] & 15u) != 0) return false;
    return true;
}

template <typename TZ>
void launch_fg_march(int sd, int mode, bool tr, const OpL0<double>& op, const TZ* z, TZ* zstore, const double* f,
                     double* out, FgState* fs, RedBuf rb, cudaStream_t s) {
    if (sd == 2) {
        if (mode == 0)
            tr ? launch_fgst_t<0, true, TZ>(op, z, zstore, f, out, fs, rb, s)
               : launch_fgst_t<0, false, TZ>(op, z, zstore, f, out, fs, rb, s);
        else
            tr ? launch_fgst_t<1, true, TZ>(op, z, zstore, f, out, fs, rb, s)
               : launch_fgst_t<1, false, TZ>(op, z, zstore, f, out, fs, rb, s);
    } else {
        if (mode == 0)
            tr ? launch_fgx3_t<0, true, TZ>(op, z, zstore, f, out, fs, rb, s)
               : launch_fgx3_t<0, false, TZ>(op, z, zstore, f, out, fs, rb, s);
        else
            tr ? launch_fgx3_t<1, true, TZ>(op, z, zstore, f, out, fs, rb, s)
               : launch_fgx3_t<1, false, TZ>(op, z, zstore, f, out, fs, rb, s);
    }
}
template void launch_fg_march<float>(int, int, bool, const OpL0<double>&, const float*, float*, const double*,
                                     double*, FgState*, RedBuf, cudaStream_t);
template void launch_fg_march<double>(int, int, bool, const OpL0<double>&, const double*, double*, const double*,
                                      double*, FgState*, RedBuf, cudaStream_t);

}  // namespace st
