// Inner eigensolve of the block-pair one-sided Jacobi: the symmetric 64 x 64
// Gram matrix G of two row blocks is diagonalised in shared memory by
// two-sided cyclic Jacobi, and the rotations are accumulated in Qt, so that
// Qt G Qt^T is diagonal and Qt Y is what one-sided Jacobi on the 64 rows Y
// of the pair would give (in exact arithmetic the two-sided rotation of G is
// the Gram matrix of the one-sided rotation of the rows).
//
// The round-robin (circle) schedule on 64 indices meets every two indices once
// per sweep in 63 rounds of 32 disjoint pairs.  One barrier per round:
//   * G is double-buffered and only its upper triangle (with the diagonal) is
//     kept, index (min, max);
//   * warps 1..7 write G after round r (each 2 x 2 block R_P B R_Q^T of the
//     pairs P < Q of the round, and the rotated diagonal blocks) into the other
//     buffer and rotate rows p, q of Qt;
//   * meanwhile warp 0 computes the rotations of round r + 1, reading the
//     three entries each needs from the buffer before round r and applying
//     round r's rotations itself with the same arithmetic as the owner of the
//     entry's block, and publishes round r + 1's pairs and the pair of each
//     index with them, so that the other warps do no index arithmetic;
//   * a round in which no pair rotates writes nothing, and the buffers stay.
// The stopping tests are those of the sweep: a pair rotates when its coupling
// g fails |g| <= tin sqrt(a b) (and is above the absolute floor); after the
// first inner sweep, couplings at the rounding level of earlier rotations
// (|g| <= 8 u max(a, b)) are left to the next outer visit.  The iteration ends
// after a sweep without rotations or after max_sweeps sweeps.
#pragma once

namespace amdd {

constexpr int JPI_N = 64;       // order of the pair's Gram matrix
constexpr int JPI_P = 32;       // disjoint pairs per round
constexpr int JPI_LDG = 65;     // G buffers, row-major (upper triangle used)
constexpr int JPI_LDQ = 68;     // Qt, row-major (16-byte aligned rows)
constexpr int JPI_THREADS = 256;

template <typename T>
struct JpRound {
    T cs[JPI_P], sn[JPI_P], a[JPI_P], b[JPI_P];
    int on[JPI_P];             // pair k rotates in this round
    int pq[JPI_P];             // pair k's indices p | q << 8
    unsigned char pos[JPI_N];  // the pair holding index x, | 0x80 for its q member
    int any;                   // some pair rotates
    int stop;                  // the iteration ends before this round
};

// pair k of round rr: indices p, q
__device__ __forceinline__ void jpi_pair(int k, int rr, int& p, int& q) {
    if (k == 0) {
        p = JPI_N - 1;
        q = rr;
    } else {
        p = (rr + k) % (JPI_N - 1);
        q = (rr - k + JPI_N - 1) % (JPI_N - 1);
    }
}

__device__ __forceinline__ float jpi_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double jpi_rsqrt(double x) { return rsqrt(x); }

__device__ __forceinline__ int jpi_gi(int x, int y) { return x < y ? x * JPI_LDG + y : y * JPI_LDG + x; }

// the 2 x 2 block of G at rows {p, q} (pair with rotation c1, s1) and columns
// {p2, q2} (rotation c2, s2) after the round: n = R_1 B R_2^T, row-major
template <typename T>
__device__ __forceinline__ void jpi_block(const T* G, int p, int q, int p2, int q2, T c1, T s1, T c2, T s2, T* n) {
    const T b00 = G[jpi_gi(p, p2)], b01 = G[jpi_gi(p, q2)];
    const T b10 = G[jpi_gi(q, p2)], b11 = G[jpi_gi(q, q2)];
    const T u00 = fma(c1, b00, -s1 * b10), u01 = fma(c1, b01, -s1 * b11);
    const T u10 = fma(s1, b00, c1 * b10), u11 = fma(s1, b01, c1 * b11);
    n[0] = fma(c2, u00, -s2 * u01);
    n[1] = fma(s2, u00, c2 * u01);
    n[2] = fma(c2, u10, -s2 * u11);
    n[3] = fma(s2, u10, c2 * u11);
}

// Rotation that makes rows p, q (Gram [[a, g], [g, b]]) orthogonal:
// t = tan(theta) is the smaller root of t^2 + 2 zeta t - 1 = 0, zeta =
// (b - a) / (2 g), written as t = sign(b - a) 2 g / (|b - a| + sqrt((b - a)^2 +
// 4 g^2)); cs = 1/sqrt(1 + t^2), sn = cs t.
template <typename T>
__device__ __forceinline__ void jpi_rotation(T a, T b, T g, T& cs, T& sn, T& t) {
    const T dd = b - a;
    const T g2 = g + g;
    t = copysign(T(1), dd) * g2 / (fabs(dd) + sqrt(fma(dd, dd, g2 * g2)));
    cs = jpi_rsqrt(fma(t, t, T(1)));
    sn = cs * t;
}

// Warp 0, lane k: the rotation of pair k of round rrn (inner sweep swn) into
// nx, with nx's pair tables, from G (the state before round rr) and round rr's
// rotations cur, which are still pending when `pend`.  Returns whether pair k
// rotates.
template <typename T>
__device__ __forceinline__ bool jpi_next(const T* G, const JpRound<T>& cur, bool pend, int rrn, int swn, T tin,
                                         T absf, T ueps, JpRound<T>& nx, int lane) {
    int p, q;
    jpi_pair(lane, rrn, p, q);
    nx.pq[lane] = p | (q << 8);
    nx.pos[p] = (unsigned char)lane;
    nx.pos[q] = (unsigned char)(lane | 0x80);
    T a, b, g;
    if (!pend) {
        a = G[p * JPI_LDG + p];
        b = G[q * JPI_LDG + q];
        g = G[jpi_gi(p, q)];
    } else {
        const int i1 = cur.pos[p], i2 = cur.pos[q];
        const int P1 = i1 & 31, P2 = i2 & 31;
        a = cur.on[P1] ? ((i1 & 0x80) ? cur.b[P1] : cur.a[P1]) : G[p * JPI_LDG + p];
        b = cur.on[P2] ? ((i2 & 0x80) ? cur.b[P2] : cur.a[P2]) : G[q * JPI_LDG + q];
        // p and q sit in different pairs of round rr; the block is taken with
        // the lower pair index as its rows, as its owner takes it
        const bool sw = P1 > P2;
        const int P = sw ? P2 : P1, Q = sw ? P1 : P2;
        const int ix = sw ? i2 : i1, iy = sw ? i1 : i2;  // the row index's and the column index's entries
        const int pqP = cur.pq[P], pqQ = cur.pq[Q];
        T n[4];
        jpi_block(G, pqP & 255, pqP >> 8, pqQ & 255, pqQ >> 8, cur.cs[P], cur.sn[P], cur.cs[Q], cur.sn[Q], n);
        const T r0 = (iy & 0x80) ? n[1] : n[0], r1 = (iy & 0x80) ? n[3] : n[2];
        g = (ix & 0x80) ? r1 : r0;
    }
    const bool doit = g != T(0) && g * g > tin * tin * a * b && fabs(g) > absf &&
                      (swn == 0 || fabs(g) > T(8) * ueps * fmax(a, b));
    nx.on[lane] = doit ? 1 : 0;
    nx.cs[lane] = T(1);
    nx.sn[lane] = T(0);
    if (doit) {
        T cs, sn, t;
        jpi_rotation(a, b, g, cs, sn, t);
        nx.cs[lane] = cs;
        nx.sn[lane] = sn;
        nx.a[lane] = fma(-t, g, a);
        nx.b[lane] = fma(t, g, b);
    }
    return doit;
}

// Four consecutive entries of a row (16-byte aligned)
__device__ __forceinline__ void jpi_ld4(const float* p, float* v) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
}
__device__ __forceinline__ void jpi_ld4(const double* p, double* v) {
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
}
__device__ __forceinline__ void jpi_st4(float* p, const float* v) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void jpi_st4(double* p, const double* v) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
}

// The blocks and Qt row segments of one of the 224 threads of warps 1..7
// (fixed over the rounds): blocks {P, Q}, P <= Q, of the 496 off-diagonal
// ones (P + 1..15 mod 32 once, P + 16 for P < 16) and the 32 diagonal ones;
// Qt tasks: pair k, columns 4 j .. 4 j + 3 (16 consecutive threads share k).
constexpr int JPI_WORKERS = JPI_THREADS - 32;
constexpr int JPI_NBLK = (528 + JPI_WORKERS - 1) / JPI_WORKERS;
constexpr int JPI_NQT = (JPI_P * 16 + JPI_WORKERS - 1) / JPI_WORKERS;

struct JpiWork {
    int blk[JPI_NBLK];  // P | Q << 8, or -1
    int qt[JPI_NQT];    // k | column << 8, or -1
};

__device__ __forceinline__ JpiWork jpi_work(int t) {
    JpiWork w;
#pragma unroll
    for (int j = 0; j < JPI_NBLK; ++j) {
        const int e = t + j * JPI_WORKERS;
        int P, Q;
        if (e < 480) {
            P = e / 15;
            Q = (P + 1 + e % 15) & (JPI_P - 1);
        } else {
            P = e < 496 ? e - 480 : e - 496;
            Q = e < 496 ? P + 16 : P;
        }
        w.blk[j] = e < 528 ? (min(P, Q) | (max(P, Q) << 8)) : -1;
    }
#pragma unroll
    for (int j = 0; j < JPI_NQT; ++j) {
        const int e = t + j * JPI_WORKERS;
        w.qt[j] = e < JPI_P * 16 ? ((e >> 4) | (((e & 15) * 4) << 8)) : -1;
    }
    return w;
}

// Warps 1..7: G after the round into Gn (from Gc and the round's rotations),
// rows of Qt rotated.
template <typename T>
__device__ __forceinline__ void jpi_apply(const T* Gc, T* Gn, T* Qt, const JpRound<T>& cur, const JpiWork& w) {
#pragma unroll
    for (int j = 0; j < JPI_NBLK; ++j) {
        const int bq = w.blk[j];
        if (bq < 0) continue;
        const int P = bq & 255, Q = bq >> 8;
        const int pqP = cur.pq[P];
        const int p = pqP & 255, q = pqP >> 8;
        if (P == Q) {
            const int gpq = jpi_gi(p, q);
            if (cur.on[P]) {
                Gn[p * JPI_LDG + p] = cur.a[P];
                Gn[q * JPI_LDG + q] = cur.b[P];
                Gn[gpq] = T(0);
            } else {
                Gn[p * JPI_LDG + p] = Gc[p * JPI_LDG + p];
                Gn[q * JPI_LDG + q] = Gc[q * JPI_LDG + q];
                Gn[gpq] = Gc[gpq];
            }
            continue;
        }
        const int pqQ = cur.pq[Q];
        const int p2 = pqQ & 255, q2 = pqQ >> 8;
        T n[4];
        jpi_block(Gc, p, q, p2, q2, cur.cs[P], cur.sn[P], cur.cs[Q], cur.sn[Q], n);
        Gn[jpi_gi(p, p2)] = n[0];
        Gn[jpi_gi(p, q2)] = n[1];
        Gn[jpi_gi(q, p2)] = n[2];
        Gn[jpi_gi(q, q2)] = n[3];
    }
#pragma unroll
    for (int j = 0; j < JPI_NQT; ++j) {
        const int tq = w.qt[j];
        if (tq < 0) continue;
        const int k = tq & 255, c = tq >> 8;
        if (!cur.on[k]) continue;
        const int pq = cur.pq[k];
        const T cs = cur.cs[k], sn = cur.sn[k];
        T* rp = Qt + (pq & 255) * JPI_LDQ + c;
        T* rq = Qt + (pq >> 8) * JPI_LDQ + c;
        T u[4], v[4], x[4], y[4];
        jpi_ld4(rp, u);
        jpi_ld4(rq, v);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            x[i] = fma(cs, u[i], -sn * v[i]);
            y[i] = fma(sn, u[i], cs * v[i]);
        }
        jpi_st4(rp, x);
        jpi_st4(rq, y);
    }
}

// The whole inner iteration.  G0 holds the pair's Gram matrix (upper triangle
// and diagonal used), G1 is scratch of the same shape, Qt the identity; jr is
// shared scratch for two rounds.  Called by all JPI_THREADS threads; returns
// (to every thread) the number of inner sweeps; *nrot_out (warp 0) counts the
// rotations.
template <typename T>
__device__ int jpi_solve(T* G0, T* G1, T* Qt, JpRound<T>* jr, T tin, T absf, int max_sweeps, unsigned& nrot_out) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const T ueps = sizeof(T) == 4 ? T(1.1920928955078125e-7) : T(2.220446049250313e-16);
    unsigned nrot = 0;
    bool swrot = false;
    const JpiWork work = jpi_work(tid - 32);  // used by warps 1..7
    if (warp == 0) {
        const bool d = jpi_next<T>(G0, jr[1], false, 0, 0, tin, absf, ueps, jr[0], lane);
        nrot += d ? 1u : 0u;
        swrot = __any_sync(0xffffffffu, d);
        if (lane == 0) {
            jr[0].any = swrot ? 1 : 0;
            jr[0].stop = 0;
        }
    }
    __syncthreads();
    T* Gc = G0;
    T* Gn = G1;
    int pc = 0, rr = 0, sw = 0;
    for (int it = 0; it < max_sweeps * (JPI_N - 1); ++it) {
        const JpRound<T>& cur = jr[pc];
        JpRound<T>& nx = jr[pc ^ 1];
        const bool pend = cur.any != 0;
        const int rrn = rr + 1 == JPI_N - 1 ? 0 : rr + 1;
        const int swn = sw + (rrn == 0 ? 1 : 0);
        if (warp == 0) {
            bool stop = false;
            if (rrn == 0) {
                stop = !swrot || swn >= max_sweeps;
                swrot = false;
            }
            const bool d = jpi_next<T>(Gc, cur, pend, rrn, swn, tin, absf, ueps, nx, lane);
            nrot += d ? 1u : 0u;
            const bool any = __any_sync(0xffffffffu, d);
            swrot = swrot || any;
            if (lane == 0) {
                nx.any = any ? 1 : 0;
                nx.stop = stop ? 1 : 0;
            }
        } else if (pend) {
            jpi_apply<T>(Gc, Gn, Qt, cur, work);
        }
        __syncthreads();
        if (pend) {
            T* s = Gc;
            Gc = Gn;
            Gn = s;
        }
        if (nx.stop) break;
        pc ^= 1;
        rr = rrn;
        sw = swn;
    }
    nrot_out = nrot;
    return sw + 1;
}

}  // namespace amdd
