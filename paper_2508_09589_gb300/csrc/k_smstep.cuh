#pragma once
// One Arnoldi step of the Jacobi-GMRES smoother (Sec. 3.2) on a stencil level (time-constant
// 2-D design) as ONE time-marching kernel, for step j:
//   u_j = s_{j-1} w_{j-1} - sum_{q<j} H[q][j-1] s_q u_q        (basis update of step j - 1)
//   w_j = A D^-1 u_j                                          (27-point stencil)
//   (w_j, u_q) for q <= j and ||u_j||^2                      (one deterministic reduction)
// A block owns a 32 x 8 tile of spatial nodes and a chunk of time planes, and takes two planes
// per iteration and per barrier, so that the 27 time-constant stencil coefficients held in
// registers serve both.  For each plane, the tile with its one-node halo (34 x 10 cells) of
// w_{j-1} and u_0 .. u_{j-1} is staged in a shared-memory ring by cp.async in 16-byte chunks:
// each halo row is copied as the aligned 16-byte chunks that cover it (10 per row in FP32), so
// a row sits at a per-row offset s (the row start's position inside its first chunk).  Lanes
// form u_j two elements at a time and write it over w_{j-1} in the ring slot, storing the
// tile-interior values to global memory once and adding their squares; the stencil reads u_j
// there two planes later, and the dots read u_q at the row's node from the same slot.  Against
// separate apply, dot and update passes this reads the basis once instead of twice and w once
// instead of twice per step.  Step 0 applies the stencil to the staged u_0.  The last block
// closes Hessenberg column j - 1 (norm, Givens rotation, breakdown test) and opens column j.
// All vectors must start on 16-byte boundaries (the launcher checks).
#include <stdint.h>

#include <mutex>

#include "k_ring.cuh"

namespace st {

// Dynamic shared memory of one block when two blocks share an SM (228 KB per SM, 1 KB reserved
// per block, about 1.5 KB of static shared memory for the reduction), and the opt-in maximum.
constexpr long long kStepTwoBlocks = 114176;
constexpr long long kStepMaxSmem = 232448;

// Ring slots of the step kernel for NQ source vectors of es-byte elements: the five planes in
// use by one iteration (the row m - 1 whose dots are due, the two planes whose stencils are
// applied, the two planes being combined) plus D pairs of planes in flight: about 16 FP32 or 8
// FP64 vector-planes, fewer where the ring would not leave room for two blocks per SM, at
// least one pair.
constexpr int step_ring_slots(int nq, int es) {
    const int vw = 16 / es;
    const long long plane = 10LL * ((vw - 1 + 34 + vw - 1) / vw) * vw;
    const long long slot = (long long)nq * plane * es;
    int d = (64 / es + 2 * nq - 1) / (2 * nq);
    if (d > 6) d = 6;
    const int fit = ((int)(kStepTwoBlocks / slot) - 5) / 2;
    if (d > fit) d = fit < 1 ? 1 : fit;
    return 5 + 2 * d;
}
constexpr long long step_smem_bytes(int nq, int es) {
    const int vw = 16 / es;
    return (long long)step_ring_slots(nq, es) * nq * 10LL * ((vw - 1 + 34 + vw - 1) / vw) * vw * es;
}

template <typename T, int NQ>
struct StepRing {
    static constexpr int VW = 16 / (int)sizeof(T);          // elements per 16-byte chunk
    static constexpr int ROWC = (VW - 1 + 34 + VW - 1) / VW;  // chunks covering 34 cells at any offset
    static constexpr int ROW = ROWC * VW;                   // staged elements per halo row
    static constexpr int PLANE = 10 * ROW;                  // one vector-plane of the tile
    static constexpr int NCH = 10 * ROWC;                   // 16-byte chunk positions per vector-plane
    static constexpr int NPAIR = PLANE / 2;                 // element pairs per plane (combine units)
    static constexpr int PW = (NPAIR + 7) / 8;              // combine pairs per warp, the same on both planes
    static constexpr bool CP1 = 2 * NCH <= 256;             // one (chunk position, plane) per copying lane
    static constexpr int CW = CP1 ? (2 * NCH + 7) / 8 : (NCH + 7) / 8;  // copy units per warp
    static_assert(PW <= 32 && CW <= 32, "one unit per lane");
    static constexpr int RING = step_ring_slots(NQ, (int)sizeof(T));
    static constexpr int D = (RING - 5) / 2;  // pairs of planes in flight
    static_assert(D >= 1, "the pipeline keeps at least one pair of planes in flight");
    static constexpr size_t smem = (size_t)step_smem_bytes(NQ, (int)sizeof(T));
};

// a0 * x - sum_q b_q y_q on a pair (packed two-lane FMAs in FP32)
template <typename T>
__device__ __forceinline__ void pair_scale(T& x0, T& x1, T a) {
    x0 *= a;
    x1 *= a;
}
template <typename T>
__device__ __forceinline__ void pair_fms(T& x0, T& x1, T c, T y0, T y1) {
    if constexpr (std::is_same<T, float>::value) {
        ffma2(x0, x1, -c, -c, y0, y1);
    } else {
        x0 -= c * y0;
        x1 -= c * y1;
    }
}

// The 27 stencil coefficients of a node and its 3 x 3 neighbourhood on one plane.  FP32
// holds both as register pairs for the packed two-lane FMA (fma.rn.f32x2): pairs (0,1),
// (2,3), (4,5), (6,7) of each 9-point part plus the ninth term apart.
template <typename T>
struct Sten {
    T c[27];
    T v[9];
    __device__ __forceinline__ T cf(int k) const { return c[k]; }
    __device__ __forceinline__ void gather(unsigned r0, unsigned r1, unsigned r2) {
        constexpr unsigned e = sizeof(T);
        v[0] = lds1<T>(r0); v[1] = lds1<T>(r0 + e); v[2] = lds1<T>(r0 + 2 * e);
        v[3] = lds1<T>(r1); v[4] = lds1<T>(r1 + e); v[5] = lds1<T>(r1 + 2 * e);
        v[6] = lds1<T>(r2); v[7] = lds1<T>(r2 + e); v[8] = lds1<T>(r2 + 2 * e);
    }
    __device__ __forceinline__ T vk(int k) const { return v[k]; }
    __device__ __forceinline__ T centre() const { return v[4]; }
    __device__ __forceinline__ T part(int pt) const {
        T s = 0;
#pragma unroll
        for (int k = 0; k < 9; ++k) s += c[pt * 9 + k] * v[k];
        return s;
    }
};
template <>
struct Sten<float> {
    float2 cp[3][4];
    float c8[3];
    float2 vp[4];
    float v8;
    __device__ __forceinline__ float cf(int k) const {
        const int pt = k / 9, r = k - pt * 9;
        return r == 8 ? c8[pt] : ((r & 1) ? cp[pt][r >> 1].y : cp[pt][r >> 1].x);
    }
    __device__ __forceinline__ void gather(unsigned r0, unsigned r1, unsigned r2) {
        vp[0].x = lds1<float>(r0); vp[0].y = lds1<float>(r0 + 4);
        vp[1].x = lds1<float>(r0 + 8); vp[1].y = lds1<float>(r1);
        vp[2].x = lds1<float>(r1 + 4); vp[2].y = lds1<float>(r1 + 8);
        vp[3].x = lds1<float>(r2); vp[3].y = lds1<float>(r2 + 4);
        v8 = lds1<float>(r2 + 8);
    }
    __device__ __forceinline__ float vk(int k) const {
        return k == 8 ? v8 : ((k & 1) ? vp[k >> 1].y : vp[k >> 1].x);
    }
    __device__ __forceinline__ float centre() const { return vp[2].x; }
    __device__ __forceinline__ float part(int pt) const { return dot9p(cp[pt], c8[pt], vp, v8); }
};

template <typename T, int NQ>
__global__ void __launch_bounds__(256, 2) km_sm_step(Geom g, const T* __restrict__ sc, const T* __restrict__ coef,
                                                     const unsigned char* __restrict__ dir,
                                                     const T* __restrict__ dinv, Ptrs<T> U,
                                                     const T* __restrict__ wprev, T* __restrict__ wout, int chunk,
                                                     int j, int steps, SmState* st_, RedBuf rb) {
    pdl_enter();
    using R = StepRing<T, NQ>;
    constexpr bool FIRST = NQ == 1;  // step 0: the stencil of u_0 itself
    constexpr int VW = R::VW, ROW = R::ROW, PLANE = R::PLANE, ROWC = R::ROWC, D = R::D, RING = R::RING;
    constexpr int M = VW - 1;  // element offset within a chunk
    constexpr unsigned ES = sizeof(T);
    constexpr unsigned SLOTB = NQ * PLANE * ES, PLANEB = PLANE * ES, ROWB = ROW * ES;
    SmStateT<T>* st = smt<T>(st_);
    if (st->stop || (FIRST ? 0 : j - 1) >= st->kdim) return;
    // [RING][NQ][10][ROW] staged source planes; vector 0 of a slot (w_{j-1}) is overwritten by
    // u_j once the plane is combined, and the stencil reads it there.  Loads and stores take
    // byte offsets (raw_s = 0); cp.async takes shared-window addresses (cwin + offset).
    constexpr unsigned raw_s = 0;
    const unsigned cwin = (unsigned)__cvta_generic_to_shared(g_step_smem);

    // node indices fit in 32 bits (the launcher checks)
    const int tx = threadIdx.x, ty = threadIdx.y;  // blockDim = (32, 8): lane tx of warp ty
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 8;
    const int i = i0 + tx, jj = j0 + ty;
    const int nt = g.net, nx1 = g.nx1, ny1 = g.ny1;
    const int n0 = blockIdx.z * chunk;
    const int n1 = min(n0 + chunk, nt + 1);
    const int ms = n0 > 0 ? n0 - 1 : 0;  // planes [ms, me] feed rows [n0, n1)
    const int me = n1 <= nt ? n1 : nt;
    const int P = nx1 * ny1;
    const int N = (int)g.nnodes;
    const bool in = i < nx1 && jj < ny1;
    const int p = in ? jj * nx1 + i : 0;

    // update coefficients (column j - 1)
    T cf[NQ > 1 ? NQ - 1 : 1];
    T a = T(1);
    if constexpr (!FIRST) {
        a = st->s[j - 1];
#pragma unroll
        for (int q = 0; q < NQ - 1; ++q) cf[q] = st->H[q * kMaxSmooth + j - 1] * st->s[q];
    }
    T* __restrict__ uj = U.p[FIRST ? 0 : j];

    // copy role, CW lanes of every warp: one chunk position of one plane of a pair (or of both
    // planes where the positions outnumber the lanes), every source vector
    const int cu = ty * R::CW + tx;
    const bool cthr = tx < R::CW && cu < (R::CP1 ? 2 * R::NCH : R::NCH);
    const int chalf = (R::CP1 && cthr) ? cu / R::NCH : 0;
    const int cpos = cthr ? cu - chalf * R::NCH : 0;
    const int ccy = cpos / ROWC, cch = cpos - (cpos / ROWC) * ROWC;
    const int cgy = j0 - 1 + ccy;
    const bool crow = cthr && cgy >= 0 && cgy < ny1;
    const int cbytes = crow ? 16 : 0;        // on planes 1 .. n_t - 1 every chunk lies inside the vector
    const int crowE = cgy * nx1 + (i0 - 1);  // element of cell x = i0 - 1 on plane 0 (may be < 0)
    const unsigned cdst = cwin + ES * (unsigned)(ccy * ROW + cch * VW);
    // combine role, PW lanes of every warp: the element pair at ue of halo row uy, on each
    // plane the block combines
    const int upi = ty * R::PW + tx;
    const bool uthr = !FIRST && tx < R::PW && upi < R::NPAIR;
    const int uy = uthr ? upi / (ROW / 2) : 0;
    const int ue = uthr ? 2 * (upi - uy * (ROW / 2)) : 0;
    const int ugy = j0 - 1 + uy;
    const bool urow_own = uthr && uy >= 1 && uy <= 8 && ugy < ny1;
    const int urowE = ugy * nx1 + (i0 - 1);
    const unsigned usrc = raw_s + ES * (unsigned)(uy * ROW + ue);
    const int uroff = urowE & M;
    // for each row offset s: which of the pair's two cells lie in the tile interior (2 bits)
    unsigned uown = 0;
#pragma unroll
    for (int sh = 0; sh < VW; ++sh)
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const int cx = ue + l - sh;  // cell column in the 34-wide halo tile
            if (cx >= 1 && cx <= 32 && i0 - 1 + cx < nx1) uown |= 1u << (2 * sh + l);
        }
    // stencil rows ty, ty + 1, ty + 2 of the halo tile: their offsets on plane 0
    int roff[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) roff[d] = ((j0 - 1 + ty + d) * nx1 + (i0 - 1)) & M;
    const unsigned gbase = raw_s + ES * (unsigned)(ty * ROW + tx);            // row ty, cell tx
    const unsigned ebase = raw_s + ES * (unsigned)((ty + 1) * ROW + tx + 1);  // the node's cell

    Sten<T> S;
    if constexpr (std::is_same<T, float>::value) {
#pragma unroll
        for (int pt = 0; pt < 3; ++pt) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                S.cp[pt][k].x = in ? sc[(long long)(pt * 9 + 2 * k) * P + p] : 0.f;
                S.cp[pt][k].y = in ? sc[(long long)(pt * 9 + 2 * k + 1) * P + p] : 0.f;
            }
            S.c8[pt] = in ? sc[(long long)(pt * 9 + 8) * P + p] : 0.f;
        }
    } else {
#pragma unroll
        for (int q = 0; q < 27; ++q) S.c[q] = in ? sc[(long long)q * P + p] : T(0);
    }
    const bool dirp = in ? (dir[p] != 0) : true;

    auto wrap = [](int k) { return k >= RING ? k - RING : k; };
    // planes m0 and m0 + 1 of the source vectors into ring slots k0 and k0 + 1; one commit
    // group per call
    auto issue = [&](int m0, int k0) {
        if (cthr) {
#pragma unroll
            for (int h = 0; h < (R::CP1 ? 1 : 2); ++h) {
                const int hh = R::CP1 ? chalf : h;
                const int mm = m0 + hh;
                if (mm <= me) {
                    const int E = mm * P + crowE;
                    const int A = (E & ~M) + cch * VW;  // chunk start (element)
                    int bytes = cbytes;
                    if (mm == 0 || mm == nt) {  // the chunk may begin before the vector or run past its end
                        bytes = 0;
                        if (crow && A >= 0 && A < N) bytes = A <= N - VW ? 16 : (N - A) * (int)ES;
                    }
                    const int Ac = bytes ? A : 0;  // a valid address when nothing is read
                    const unsigned d = cdst + (unsigned)(hh ? wrap(k0 + 1) : k0) * SLOTB;
#pragma unroll
                    for (int v = 0; v < NQ; ++v) {
                        const T* src = v == 0 ? (FIRST ? U.p[0] : wprev) : U.p[v - 1];
                        cp_async16(d + (unsigned)v * PLANEB, src + Ac, bytes);
                    }
                }
            }
        }
        cp_async_commit();
    };
    T nrm = T(0);
    // u_j of plane mm (ring slot k) at this lane's pair, written over w_{j-1} in the slot; own:
    // the plane is in this block's range (the pair's tile-interior cells then go to global
    // memory and into ||u_j||^2)
    auto combine = [&](int mm, int k, bool own) {
        if (!uthr) return;
        const unsigned sl = usrc + (unsigned)k * SLOTB;
        T x0, x1;
        lds2<T>(sl, x0, x1);
        pair_scale(x0, x1, a);
#pragma unroll
        for (int q = 0; q < NQ - 1; ++q) {
            T y0, y1;
            lds2<T>(sl + (unsigned)(1 + q) * PLANEB, y0, y1);
            pair_fms(x0, x1, cf[q], y0, y1);
        }
        if (own && urow_own) {
            const int qm = mm * P;
            const int s = (qm + uroff) & M;
            const unsigned o = (uown >> (2 * s)) & 3u;
            T* dst = uj + (qm + urowE - s + ue);  // the pair's first element
            if (o == 3u) {
                if constexpr (sizeof(T) == 4)
                    *reinterpret_cast<float2*>(dst) = make_float2(x0, x1);
                else
                    *reinterpret_cast<double2*>(dst) = make_double2(x0, x1);
                nrm += x0 * x0 + x1 * x1;
            } else {
                if (o & 1u) {
                    dst[0] = x0;
                    nrm += x0 * x0;
                }
                if (o & 2u) {
                    dst[1] = x1;
                    nrm += x1 * x1;
                }
            }
        }
        sts2<T>(sl, x0, x1);
    };
    T acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = T(0);
    // w of a row at node qn, u_j there = uc: write it, add its dots with u_0 .. u_j (u_q read
    // from ring slot k at the node's cell, shifted by the row offset s1)
    auto emit = [&](int qn, T wv, T uc, int k, int s1) {
        wout[qn] = wv;
        if constexpr (!FIRST) {
            const unsigned own = ebase + (unsigned)k * SLOTB + ES * (unsigned)s1;
#pragma unroll
            for (int q = 0; q < NQ - 1; ++q) acc[q] += wv * lds1<T>(own + (unsigned)(1 + q) * PLANEB);
        }
        acc[NQ - 1] += wv * uc;
    };
    // the 3 x 3 neighbourhood of the node on the u_j of a plane (slot k, offset mp)
    auto gather = [&](int k, int mp) {
        const unsigned base = gbase + (unsigned)k * SLOTB;
        S.gather(base + ES * (unsigned)((mp + roff[0]) & M), base + ROWB + ES * (unsigned)((mp + roff[1]) & M),
                 base + 2 * ROWB + ES * (unsigned)((mp + roff[2]) & M));
    };
    // plane gp (slot kg; slot kq holds plane gp - 1) near a boundary of the block's range or of
    // the time axis: its three row parts, the emission of row gp - 1 and, on the last plane, of
    // row n_t, with every test of the general case
    auto plane_general = [&](int gp, int kg, int kq, T& a_prev, T& a_cur, T& a_next, T c_prev, T& c_cur) {
        const int qg = gp * P;
        const int mpg = qg & M;
        gather(kg, mpg);
        c_cur = S.centre();
        if (gp >= 3 && gp + 2 <= nt) {  // rows gp - 1, gp, gp + 1 interior: scaled interior stencil
            a_next = S.part(0);
            a_cur += S.part(1);
            a_prev += S.part(2);
        } else {
            T v[9];
            const T* dm = dinv + qg;
#pragma unroll
            for (int dj = 0; dj < 3; ++dj)
#pragma unroll
                for (int di = 0; di < 3; ++di) {
                    const int ii = i + di - 1, jn = jj + dj - 1;
                    const bool ok = in && ii >= 0 && ii < nx1 && jn >= 0 && jn < ny1;
                    v[dj * 3 + di] = ok ? S.vk(dj * 3 + di) * dm[jn * nx1 + ii] : T(0);
                }
#pragma unroll
            for (int part = 0; part < 3; ++part) {
                const int r = gp + 1 - part;
                T sum = 0;
                if (r >= 1 && r <= nt) {
                    const int cl = (r == 1) ? (nt == 1 ? 3 : 0) : (r == nt ? 2 : 1);
                    const T* cc = coef + (long long)(cl * 27 + part * 9) * P + p;
#pragma unroll
                    for (int k = 0; k < 9; ++k) sum += cc[(long long)k * P] * v[k];
                }
                if (part == 0)
                    a_next = sum;
                else if (part == 1)
                    a_cur += sum;
                else
                    a_prev += sum;
            }
        }
        if (in && gp - 1 >= n0 && gp - 1 < n1) {
            const int qn = qg - P + p;
            emit(qn, (gp - 1 == 0 || dirp) ? c_prev * dinv[qn] : a_prev, c_prev, kq, (((qg - P) & M) + roff[1]) & M);
        }
        if (in && gp == nt && nt >= n0 && nt < n1) {
            const int qn = qg + p;
            emit(qn, dirp ? c_cur * dinv[qn] : a_cur, c_cur, kg, (mpg + roff[1]) & M);
        }
    };

    // prologue: planes ms .. ms + 2 D + 1 in D + 1 groups, the first pair combined
#pragma unroll
    for (int d = 0; d <= D; ++d) issue(ms + 2 * d, 2 * d);
    cp_async_wait<D>();
    __syncthreads();
    if constexpr (!FIRST) {
        combine(ms, 0, ms >= n0 && ms < n1);
        if (ms + 1 <= me) combine(ms + 1, 1, ms + 1 >= n0 && ms + 1 < n1);
    }
    // two planes m, m + 1 per iteration (one barrier): apply the stencil on planes m and m + 1,
    // emit rows m - 1 and m, combine planes m + 2 and m + 3.  Carried: aL (row m - 1, lower
    // and own parts), aM (row m, lower part), cL (u_j of row m - 1 at the node).  Lean
    // iterations: rows m - 1 .. m + 2 interior, rows m - 1 and m in range, planes m + 2 and
    // m + 3 staged and in range, no last-row emission: no tests beyond the thread's own.
    const int ml = max(n0 + 1, 3), mh = min(n1 - 1, nt) - 3;
    T aL = T(0), aM = T(0), cL = T(0);
    int m = ms, km = 0;  // km: ring slot of plane m
    while (m <= me) {
        cp_async_wait<D - 1>();  // this thread's copies of planes m + 2, m + 3 have landed
        __syncthreads();
        const int k1 = wrap(km + 1), k2 = wrap(km + 2), k3 = wrap(km + 3), kp = wrap(km + RING - 1);
        issue(m + 2 + 2 * D, wrap(km + 2 + 2 * D));  // into the slots of planes m - 3, m - 2
        T aN = T(0), aN2 = T(0), cM = T(0), cN = T(0);
        if (m >= ml && m <= mh) {
            const int qm = m * P;
            const int mp = qm & M, mp1 = (qm + P) & M, mpp = (qm - P) & M;
            gather(km, mp);
            cM = S.centre();
            aN = S.part(0);
            aM += S.part(1);
            aL += S.part(2);
            if (in) emit(qm - P + p, aL, cL, kp, (mpp + roff[1]) & M);
            gather(k1, mp1);
            cN = S.centre();
            aN2 = S.part(0);
            aN += S.part(1);
            aM += S.part(2);
            if (in) emit(qm + p, aM, cM, km, (mp + roff[1]) & M);
            if constexpr (!FIRST) {  // after the loads of this iteration's other slots
                combine(m + 2, k2, true);
                combine(m + 3, k3, true);
            }
        } else {
            plane_general(m, km, kp, aL, aM, aN, cL, cM);
            if (m + 1 <= me) plane_general(m + 1, k1, km, aM, aN, aN2, cM, cN);
            if constexpr (!FIRST) {
                if (m + 2 <= me) combine(m + 2, k2, m + 2 >= n0 && m + 2 < n1);
                if (m + 3 <= me) combine(m + 3, k3, m + 3 >= n0 && m + 3 < n1);
            }
        }
        aL = aN;
        aM = aN2;
        cL = cN;
        m += 2;
        km = k2;
    }
    cp_async_wait<0>();

    // one reduction: the NQ dots and, after step 0, ||u_j||^2
    constexpr int NR = FIRST ? 1 : NQ + 1;
    T red[NR];
#pragma unroll
    for (int q = 0; q < NQ; ++q) red[q] = acc[q];
    if constexpr (!FIRST) red[NQ] = nrm;
    __shared__ double out[NR];
    if (reduce_publish_t<T, NR>(red, NR, rb, out)) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            if constexpr (FIRST) {
                sm_apply_finish<T>(st_, out, 0);
            } else {
                sm_update_finish<T>(st_, out[NQ], j - 1, steps);  // closes column j - 1
                if (j < st->kdim) sm_apply_finish<T>(st_, out, j);  // opens column j
            }
        }
    }
}

template <typename T, int NQ>
static void launch_sm_step_nq(const Geom& g, const T* sc, const T* coef, const unsigned char* dir, const T* dinv,
                              const Ptrs<T>& U, const T* wprev, T* wout, int j, int steps, SmState* st, RedBuf rb,
                              cudaStream_t s) {
    dim3 grid, block;
    const MarchGrid mg = march_grid(g, grid, block);
    constexpr size_t bytes = StepRing<T, NQ>::smem;
    static std::once_flag attr;  // once per instantiation (server slot threads reach this together)
    std::call_once(attr, [] {
        cudaFuncSetAttribute(km_sm_step<T, NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    });
    launch_pdl(km_sm_step<T, NQ>, grid, block, bytes, s, g, sc, coef, dir, dinv, U, wprev, wout, mg.chunk, j, steps,
               st, rb);
}

// The vectors the step kernel stages or stores with 16-byte copies must start on 16-byte
// boundaries, the level must have fewer than 2^31 nodes and at least 64 per plane, and the ring
// of every step must fit in one block's shared memory; the caller uses the separate kernels
// otherwise.
template <typename T>
bool sm_step_aligned(const Ptrs<T>& U, int steps, const T* w, const T* w2, long long nnodes, long long plane) {
    if (nnodes > (1LL << 31) - 64) return false;  // the kernel indexes nodes in 32 bits
    if (plane < 64) return false;  // the chunks of a plane's last halo row end inside the next plane
    for (int nq = 1; nq <= steps; ++nq)
        if (step_smem_bytes(nq, (int)sizeof(T)) > kStepMaxSmem) return false;  // ring beyond one block's limit
    auto ok = [](const void* q) { return ((uintptr_t)q & 15u) == 0; };
    if (!ok(w) || !ok(w2)) return false;
    for (int q = 0; q <= steps; ++q)
        if (!ok(U.p[q])) return false;
    return true;
}

template <typename T>
void launch_sm_step(const Geom& g, const T* sc, const T* coef, const unsigned char* dir, const T* dinv,
                    const Ptrs<T>& U, const T* wprev, T* wout, int j, int steps, SmState* st, RedBuf rb,
                    cudaStream_t s) {
    note_launch(s);
#define ST_STEP_CASE(NQv) \
    case NQv:             \
        launch_sm_step_nq<T, NQv>(g, sc, coef, dir, dinv, U, wprev, wout, j, steps, st, rb, s); \
        break;
    switch (j + 1) {
        ST_STEP_CASE(1)
        ST_STEP_CASE(2)
        ST_STEP_CASE(3)
        ST_STEP_CASE(4)
        ST_STEP_CASE(5)
        ST_STEP_CASE(6)
        ST_STEP_CASE(7)
        ST_STEP_CASE(8)
        ST_STEP_CASE(9)
        ST_STEP_CASE(10)
        ST_STEP_CASE(11)
        ST_STEP_CASE(12)
        ST_STEP_CASE(13)
        ST_STEP_CASE(14)
        ST_STEP_CASE(15)
        ST_STEP_CASE(16)
        default:
            break;
    }
#undef ST_STEP_CASE
}

}  // namespace st
