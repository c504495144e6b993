#pragma once
// One Arnoldi step of the Jacobi-GMRES smoother (Sec. 3.2) on a stencil level (time-constant
// 2-D design) as ONE time-marching kernel, for step j:
//   u_j = s_{j-1} w_{j-1} - sum_{q<j} H[q][j-1] s_q u_q        (basis update of step j - 1)
//   w_j = A D^-1 u_j                                          (27-point stencil)
//   (w_j, u_q) for q <= j and ||u_j||^2                      (one deterministic reduction)
// A block owns a 32 x 8 tile of spatial nodes and a chunk of time planes.  For each plane,
// the tile with its one-node halo (34 x 10 cells) of w_{j-1} and u_0 .. u_{j-1} is staged in
// shared memory by cp.async in 16-byte chunks: each halo row is copied as the aligned
// 16-byte chunks that cover it (10 per row in FP32), so a row sits at a per-row offset s
// (the row start's position inside its first chunk).  Threads form u_j two elements at a
// time into a staging buffer, writing the tile-interior values to global memory once and
// adding their squares; the stencil reads u_j from that buffer, and the dots read u_q at the
// row's node from the staged ring.  Against separate apply, dot and update passes this reads
// the basis once instead of twice and w once instead of twice per step.  Step 0 applies the
// stencil to u_0 and takes (w_0, u_0).  The last block closes Hessenberg column j - 1 (norm,
// Givens rotation, breakdown test) and opens column j.  All vectors must start on 16-byte
// boundaries (the launcher checks).
#include <stdint.h>

#include <mutex>

#include "st_device.cuh"

namespace st {

template <typename T, int NQ>
struct StepRing {
    static constexpr int VW = 16 / (int)sizeof(T);          // elements per 16-byte chunk
    static constexpr int ROWC = (VW - 1 + 34 + VW - 1) / VW;  // chunks covering 34 cells at any offset
    static constexpr int ROW = ROWC * VW;                   // staged elements per halo row
    static constexpr int PLANE = 10 * ROW;                  // one vector-plane of the tile
    static constexpr int NCH = 10 * ROWC;                   // 16-byte chunk positions per vector-plane
    static constexpr int NPAIR = PLANE / 2;                 // element pairs per plane (combine units)
    static constexpr int NPAR = 2 * NCH <= 256 ? 2 : 1;     // threads sharing one chunk position's copies
    // ring of RING plane slots: PF = RING - 2 planes issued ahead (PF - 1 in flight while a
    // plane is consumed: about 16 FP32 or 8 FP64 vector-planes per block, within 110 KB so that
    // two blocks share an SM), plus the plane being combined and the one whose dots are due
    static constexpr int K = 64 / (int)sizeof(T);
    static constexpr int want = 3 + (K + NQ - 1) / NQ;
    static constexpr size_t slot_bytes = (size_t)NQ * PLANE * sizeof(T);
    static constexpr int fit = (int)((110u * 1024u - 2 * PLANE * sizeof(T)) / slot_bytes);  // 2 blocks per SM
    static constexpr int RING0 = want > 16 ? 16 : want;
    static constexpr int RING1 = RING0 > fit ? fit : RING0;
    static constexpr int RING = RING1 < 4 ? 4 : RING1;  // at least 2 planes in flight
    static constexpr int PF = RING - 2;
    static_assert(PF >= 2, "the pipeline waits for the plane after the current one");
    static constexpr size_t smem = sizeof(T) * ((size_t)RING * NQ * PLANE + 2 * PLANE);
};

template <typename T>
struct Pair;
template <>
struct Pair<float> {
    using V = float2;
};
template <>
struct Pair<double> {
    using V = double2;
};

__device__ __forceinline__ void cp_async16(unsigned smem_dst, const void* gsrc, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_dst), "l"(gsrc), "r"(src_bytes)
                 : "memory");
}

// Shared-memory accesses by 32-bit shared-window address (ld/st.shared), one or two elements.
template <typename T>
__device__ __forceinline__ T lds1(unsigned a) {
    T v;
    if constexpr (sizeof(T) == 4)
        asm volatile("ld.shared.f32 %0, [%1];\n" : "=f"(v) : "r"(a) : "memory");
    else
        asm volatile("ld.shared.f64 %0, [%1];\n" : "=d"(v) : "r"(a) : "memory");
    return v;
}
template <typename T>
__device__ __forceinline__ void lds2(unsigned a, T& x, T& y) {
    if constexpr (sizeof(T) == 4)
        asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];\n" : "=f"(x), "=f"(y) : "r"(a) : "memory");
    else
        asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];\n" : "=d"(x), "=d"(y) : "r"(a) : "memory");
}
template <typename T>
__device__ __forceinline__ void sts2(unsigned a, T x, T y) {
    if constexpr (sizeof(T) == 4)
        asm volatile("st.shared.v2.f32 [%0], {%1, %2};\n" ::"r"(a), "f"(x), "f"(y) : "memory");
    else
        asm volatile("st.shared.v2.f64 [%0], {%1, %2};\n" ::"r"(a), "d"(x), "d"(y) : "memory");
}

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
    constexpr int VW = R::VW, ROW = R::ROW, PLANE = R::PLANE, ROWC = R::ROWC, PF = R::PF, RING = R::RING;
    constexpr int M = VW - 1;  // element offset within a chunk
    constexpr unsigned ES = sizeof(T);
    constexpr unsigned SLOTB = NQ * PLANE * ES, PLANEB = PLANE * ES, ROWB = ROW * ES;
    SmStateT<T>* st = smt<T>(st_);
    if (st->stop || (FIRST ? 0 : j - 1) >= st->kdim) return;
    extern __shared__ __align__(16) unsigned char smem_bytes[];
    // [RING][NQ][10][ROW] staged source planes, then [2][10][ROW] u_j of the current and next plane
    const unsigned raw_s = (unsigned)__cvta_generic_to_shared(smem_bytes);
    const unsigned stg_s = raw_s + RING * SLOTB;

    // node indices fit in 32 bits (the launcher checks)
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
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
    const int pstep = P & M;  // row offsets advance by P mod VW per plane

    // update coefficients (column j - 1)
    T cf[NQ > 1 ? NQ - 1 : 1];
    T a = T(1);
    if constexpr (!FIRST) {
        a = st->s[j - 1];
#pragma unroll
        for (int q = 0; q < NQ - 1; ++q) cf[q] = st->H[q * kMaxSmooth + j - 1] * st->s[q];
    }
    T* __restrict__ uj = U.p[FIRST ? 0 : j];

    // copy role: chunk position cpos of halo row ccy (threads < NPAR * NCH), every NPAR-th vector
    const bool cthr = tid < R::NPAR * R::NCH;
    const int cpar = cthr ? tid / R::NCH : 0;
    const int cpos = cthr ? tid - cpar * R::NCH : 0;
    const int ccy = cpos / ROWC, cch = cpos - (cpos / ROWC) * ROWC;
    const int cgy = j0 - 1 + ccy;
    const bool crow = cthr && cgy >= 0 && cgy < ny1;
    const int cbytes = crow ? 16 : 0;        // on planes 1 .. n_t - 1 every chunk lies inside the vector
    const int crowE = cgy * nx1 + (i0 - 1);  // element of cell x = i0 - 1 on plane 0 (may be < 0)
    const unsigned cdst = raw_s + ES * (unsigned)(ccy * ROW + cch * VW);
    // combine role: element pair at ue of halo row uy (threads < NPAIR)
    const bool uthr = tid < R::NPAIR;
    const int uy = uthr ? tid / (ROW / 2) : 0;
    const int ue = uthr ? 2 * (tid - uy * (ROW / 2)) : 0;
    const int ugy = j0 - 1 + uy;
    const bool urow_own = uthr && uy >= 1 && uy <= 8 && ugy < ny1;
    const int urowE = ugy * nx1 + (i0 - 1);
    const unsigned usrc = raw_s + ES * (unsigned)(uy * ROW + ue);
    const unsigned udst = stg_s + ES * (unsigned)(uy * ROW + ue);
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
    const unsigned gbase = stg_s + ES * (unsigned)(ty * ROW + tx);         // row ty, cell tx
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
    // plane m (first element qm = m P) of the source vectors into ring slot k; one commit
    // group per call
    auto issue = [&](int m, int qm, int k) {
        if (m <= me && cthr) {
            const int E = qm + crowE;
            const int A = (E & ~M) + cch * VW;  // chunk start (element)
            int bytes = cbytes;
            if (m == 0 || m == nt) {  // the chunk may begin before the vector or run past its end
                bytes = 0;
                if (crow && A >= 0 && A < N) bytes = A <= N - VW ? 16 : (N - A) * (int)ES;
            }
            const int Ac = bytes ? A : 0;  // a valid address when nothing is read
            const unsigned d = cdst + (unsigned)k * SLOTB;
            auto copy = [&](auto first) {
                constexpr int v0 = decltype(first)::value;
#pragma unroll
                for (int v = v0; v < NQ; v += R::NPAR) {
                    const T* src = v == 0 ? (FIRST ? U.p[0] : wprev) : U.p[v - 1];
                    cp_async16(d + (unsigned)v * PLANEB, src + Ac, bytes);
                }
            };
            if (R::NPAR == 1 || cpar == 0)
                copy(std::integral_constant<int, 0>{});
            else
                copy(std::integral_constant<int, 1>{});
        }
        cp_async_commit();
    };
    T nrm = T(0);
    // u_j of plane m (first element qm, offset mp) from slot k into stg buffer b at this
    // thread's pair; own: the plane is in this block's range (the pair's tile-interior cells
    // are then written to global memory)
    auto combine = [&](int qm, int mp, int k, int b, bool own) {
        if (!uthr) return;
        const unsigned sl = usrc + (unsigned)k * SLOTB;
        T x0, x1;
        lds2<T>(sl, x0, x1);
        if constexpr (!FIRST) {
            pair_scale(x0, x1, a);
#pragma unroll
            for (int q = 0; q < NQ - 1; ++q) {
                T y0, y1;
                lds2<T>(sl + (unsigned)(1 + q) * PLANEB, y0, y1);
                pair_fms(x0, x1, cf[q], y0, y1);
            }
            if (own && urow_own) {
                const int s = (mp + uroff) & M;
                const unsigned o = (uown >> (2 * s)) & 3u;
                const bool o0 = o & 1u, o1 = o & 2u;
                T* dst = uj + (qm + urowE - s + ue);  // the pair's first element
                if (o == 3u) {
                    if constexpr (sizeof(T) == 4)
                        *reinterpret_cast<float2*>(dst) = make_float2(x0, x1);
                    else
                        *reinterpret_cast<double2*>(dst) = make_double2(x0, x1);
                    nrm += x0 * x0 + x1 * x1;
                } else {
                    if (o0) {
                        dst[0] = x0;
                        nrm += x0 * x0;
                    }
                    if (o1) {
                        dst[1] = x1;
                        nrm += x1 * x1;
                    }
                }
            }
        }
        sts2<T>(udst + (unsigned)b * PLANEB, x0, x1);
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
    // the 3 x 3 neighbourhood of the node on the staged u_j of a plane (buffer b, offset mp)
    auto gather = [&](int b, int mp) {
        const unsigned base = gbase + (unsigned)b * PLANEB;
        S.gather(base + ES * (unsigned)((mp + roff[0]) & M), base + ROWB + ES * (unsigned)((mp + roff[1]) & M),
                 base + 2 * ROWB + ES * (unsigned)((mp + roff[2]) & M));
    };

    // running plane state: m, its first element qm = m P, offset mp = qm mod VW, ring slot km
    int m = ms, km = 0, qm = ms * P;
    int mp = qm & M;
    {
        int q = qm, mm = ms;
#pragma unroll
        for (int d = 0; d < PF; ++d) {
            issue(mm, q, d);
            ++mm;
            q += P;
        }
    }
    cp_async_wait<PF - 1>();
    __syncthreads();
    combine(qm, mp, 0, ms & 1, ms >= n0 && ms < n1);
    // lean planes: rows m - 1, m, m + 1 interior, row m - 1 in range, plane m + 1 staged and in
    // this block's range, no last-row emission: no tests beyond the thread's own
    const int ml = max(n0 + 1, 3), mh = min(min(me - 1, nt - 2), n1 - 2);
    T A = 0, B = 0, Cc = 0, E0 = 0, E1 = 0, E2 = 0;
    int mp_prev = (mp - pstep) & M;  // offset of plane m - 1
    // plane m: wait for plane m + 1, refill, stage u_j of plane m + 1, stencil plane m, emit
    auto step = [&](T& a_prev, T& a_cur, T& a_next, T& c_prev, T& c_cur) {
        cp_async_wait<PF - 2>();
        __syncthreads();
        const int k1 = wrap(km + 1), kp = wrap(km + RING - 1);
        const int mp1 = (mp + pstep) & M;
        issue(m + PF, qm + PF * P, wrap(km + PF));
        if (m >= ml && m <= mh) {
            combine(qm + P, mp1, k1, (m + 1) & 1, true);
            gather(m & 1, mp);
            c_cur = S.centre();
            a_next = S.part(0);
            a_cur += S.part(1);
            a_prev += S.part(2);
            if (in) emit(qm - P + p, a_prev, c_prev, kp, (mp_prev + roff[1]) & M);
        } else {
            if (m + 1 <= me) combine(qm + P, mp1, k1, (m + 1) & 1, m + 1 >= n0 && m + 1 < n1);
            gather(m & 1, mp);
            c_cur = S.centre();
            if (m >= 3 && m + 2 <= nt) {  // rows m - 1, m, m + 1 interior: scaled interior stencil
                a_next = S.part(0);
                a_cur += S.part(1);
                a_prev += S.part(2);
            } else {
                T v[9];
                const T* dm = dinv + qm;
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
                    const int r = m + 1 - part;
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
            if (in && m - 1 >= n0 && m - 1 < n1) {
                const int qn = qm - P + p;
                emit(qn, (m - 1 == 0 || dirp) ? c_prev * dinv[qn] : a_prev, c_prev, kp, (mp_prev + roff[1]) & M);
            }
            if (in && m == nt && nt >= n0 && nt < n1) {
                const int qn = qm + p;
                emit(qn, dirp ? c_cur * dinv[qn] : a_cur, c_cur, km, (mp + roff[1]) & M);
            }
        }
        // advance to plane m + 1
        ++m;
        qm += P;
        km = k1;
        mp_prev = mp;
        mp = mp1;
    };
    while (m <= me) {
        step(A, B, Cc, E0, E1);
        if (m > me) break;
        step(B, Cc, A, E1, E2);
        if (m > me) break;
        step(Cc, A, B, E2, E0);
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
        if (tid == 0) {
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
// boundaries and the level must have fewer than 2^31 nodes; the caller uses the separate
// kernels otherwise.
template <typename T>
bool sm_step_aligned(const Ptrs<T>& U, int steps, const T* w, const T* w2, long long nnodes) {
    if (nnodes > (1LL << 31) - 64) return false;  // the kernel indexes nodes in 32 bits
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
