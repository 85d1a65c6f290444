// Steps (II)-(III) of the assembly (Sec. 2.3): exact clipping of one P1 simplex
// against one axis-aligned Q1 cell and the integrals
//     block[a][b] = ∫_{E∩C} lambda_a psi_b,     vol = |E∩C|,
// lambda_a = barycentric coordinate a of the element, psi_b = Q1 function of
// cell corner b (bits x, y, z).
//
// Formulation (device code; the oracle uses a different one):
//  * Work in cell-local coordinates t = (x - cell_lo) / h, the cell is [0,1]^d.
//  * The boundary of P = E ∩ C consists of the element faces clipped to the
//    cell (Sutherland-Hodgman against the cell planes the element crosses) and
//    the cell faces clipped to the element (against the d+1 planes
//    lambda_a = 0).  Every boundary polygon is fanned into triangles
//    (segments in 2-D) and coned to an apex A, which turns the polytope into
//    signed simplices (divergence theorem).  In 3-D, A lies on one crossed
//    cell plane of every axis the element crosses (so the cones over those
//    cell faces have zero volume and the faces drop out) and at the centre of
//    the overlap of the element's bounding box with the cell along the other
//    axes; an element inside the cell takes one of its vertices (the element
//    faces through it drop out).  In 2-D the clipped polygon is fanned from
//    its first vertex.
//  * On each cone simplex (0, p, q[, r]) in u = t - A the monomial moments
//    needed for lambda_a psi_b (u^S and u_j u^S, S a subset of the axes) are
//    exact closed forms: for a simplex T and monomial prod_j u_{k_j} of degree
//    q, ∫_T = |T| n!/(n+q)! sum over permutations sigma of S_q of
//    prod over cycles c of sigma of (sum over vertices v of prod_{j in c} v_{k_j}).
//  * Geometry (plane tests, intersection points) is always FP64; the moment
//    arithmetic runs in R = double (FP64 mode) or R = float (mixed mode).
#pragma once

#include <climits>

#include "l2x_fp.cuh"
#include "l2x_internal.cuh"

namespace l2x {

constexpr int kMaxPoly = 9;  // one vertex added per cut: triangle + 6 planes -> 9; square + 4 planes -> 8
// doubles of one thread's polygon buffers in shared memory: 2 * kMaxPoly
// vertices plus one pad (an odd stride keeps a warp's accesses conflict-free)
template <int D>
struct PolySlot {
    static constexpr int kDoubles = 2 * kMaxPoly * D + 1;
};

template <int D>
struct ElemT {
    double T[D + 1][D];   // vertices in cell-local coordinates
};

// Sutherland-Hodgman clipping of a convex polygon against one half-space.  The
// inside vertices of a convex polygon cut by a plane form one cyclic run, so the
// output is that run with the crossing point of the exit edge (inside ->
// outside) after its last vertex and that of the entry edge before its first: a
// cut adds at most one vertex.  The crossing on edge (p, q) is p + t (q - p),
// t = s_p / (s_p - s_q), s the signed plane values; a warp computes the two
// crossings together.
//
// Rounding can split the computed inside flags into several runs, but only
// through vertices within rounding distance of the plane (the signed value of a
// convex polygon is unimodal along its boundary, so a vertex between two outside
// runs, or in an outside run that does not hold the farthest vertex, is within
// rounding of the plane).  Such a split is repaired: the outside run holding the
// vertex farthest outside is kept and the vertices of the other outside runs are
// counted inside, which moves the polygon by rounding only and keeps the bound of
// one added vertex per cut; t is then clamped to [0, 1].  So a triangle cut by the
// six cell planes, or a cell face cut by the four element planes, fits kMaxPoly.

// Emits the clipped polygon: inside vertices of `in`, crossing points X0 (after
// vertex e0) and X1 (after vertex e1).
template <int D>
__device__ __forceinline__ int clip_emit(const double (*in)[D], int n, unsigned inside, int e0, const double* X0,
                                         int e1, const double* X1, double (*out)[D]) {
    int m = 0;
    for (int i = 0; i < n; ++i) {
        if ((inside >> i) & 1u) {
#pragma unroll
            for (int j = 0; j < D; ++j) out[m][j] = in[i][j];
            ++m;
        }
        if (i == e0 || i == e1) {
            const double* X = i == e0 ? X0 : X1;
#pragma unroll
            for (int j = 0; j < D; ++j) out[m][j] = X[j];
            ++m;
        }
    }
    return m;
}

// Exit and entry edges of a single run of inside vertices (bit i = vertex i);
// false if the inside vertices do not form exactly one cyclic run.
__device__ __forceinline__ bool one_run(unsigned inside, int n, int& e_exit, int& e_entry) {
    const unsigned all = (1u << n) - 1u;
    const unsigned next = ((inside >> 1) | (inside << (n - 1))) & all;  // bit i = inside[i+1]
    const unsigned ex = inside & ~next, en = ~inside & next & all;
    if (__popc(ex) != 1 || __popc(en) != 1) return false;
    e_exit = __ffs(ex) - 1;
    e_entry = __ffs(en) - 1;
    return true;
}

// Repaired inside mask: everything but the cyclic run of outside vertices that
// holds vertex j (bit j of `outside` set; at least one bit of the n clear).
__device__ __forceinline__ unsigned keep_outside_run(unsigned outside, int n, int j) {
    unsigned run = 1u << j;
    for (int i = j + 1 == n ? 0 : j + 1; (outside >> i) & 1u; i = i + 1 == n ? 0 : i + 1) run |= 1u << i;
    for (int i = j == 0 ? n - 1 : j - 1; ((outside >> i) & 1u) && !((run >> i) & 1u); i = i == 0 ? n - 1 : i - 1)
        run |= 1u << i;
    return ((1u << n) - 1u) & ~run;
}

__device__ __forceinline__ double clamp01(double t) { return fmin(fmax(t, 0.0), 1.0); }  // NaN -> 0

// Against an axis plane at coordinate c: keep v[k] >= c (upper = false) or
// v[k] <= c (upper = true).  Inside tests are integer comparisons of order keys;
// crossing points are snapped onto the plane.  `same` is set when every vertex
// is inside: then `out` is left untouched and the polygon is `in` as it was.
template <int D, bool kFastDiv>
__device__ __forceinline__ int clip_axis(const double (*in)[D], int n, double (*out)[D], int k, double c,
                                         bool upper, bool& same) {
    const long long kc = order_key(c);
    unsigned inside = 0;
    for (int i = 0; i < n; ++i) {
        const long long kk = order_key(in[i][k]);
        inside |= (unsigned)(upper ? kk <= kc : kk >= kc) << i;
    }
    const unsigned all = (1u << n) - 1u;
    same = inside == all;
    if (same) return n;
    if (inside == 0) return 0;
    int e0, e1;
    const bool repaired = !one_run(inside, n, e0, e1);
    if (repaired) {
        int j = -1;
        long long kj = 0;
        for (int i = 0; i < n; ++i) {
            if ((inside >> i) & 1u) continue;
            const long long kk = order_key(in[i][k]);
            if (j < 0 || (upper ? kk > kj : kk < kj)) { j = i; kj = kk; }
        }
        inside = keep_outside_run(~inside & all, n, j);
        one_run(inside, n, e0, e1);
    }
    // both quotients before the one branch, so that their latencies overlap
    double t[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int i = r == 0 ? e0 : e1;
        const double* p = in[i];
        const double* q = in[i + 1 == n ? 0 : i + 1];
        t[r] = kFastDiv ? div_fast(p[k] - c, p[k] - q[k]) : div_nr(p[k] - c, p[k] - q[k]);
    }
    if (repaired) {
        t[0] = clamp01(t[0]);
        t[1] = clamp01(t[1]);
    }
    double X[2][D];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int i = r == 0 ? e0 : e1;
        const double* p = in[i];
        const double* q = in[i + 1 == n ? 0 : i + 1];
        // the coordinate on the plane is the plane's (snapped); only the other
        // axes interpolate, placed by integer selects
        if constexpr (D == 3) {
            const int j1 = k == 0 ? 1 : 0, j2 = k == 2 ? 1 : 2;
            const double v1 = fma(t[r], q[j1] - p[j1], p[j1]);
            const double v2 = fma(t[r], q[j2] - p[j2], p[j2]);
            X[r][0] = k == 0 ? c : v1;
            X[r][1] = k == 1 ? c : (k == 0 ? v1 : v2);
            X[r][2] = k == 2 ? c : v2;
        } else {
            const double v1 = fma(t[r], q[1 - k] - p[1 - k], p[1 - k]);
            X[r][0] = k == 0 ? c : v1;
            X[r][1] = k == 1 ? c : v1;
        }
    }
    return clip_emit<D>(in, n, inside, e0, X[0], e1, X[1], out);
}

// Against the half-space g.v + c0 >= 0 (`same` as for clip_axis).
template <int D, bool kFastDiv>
__device__ __forceinline__ int clip_plane(const double (*in)[D], int n, double (*out)[D], const double* g,
                                          double c0, bool& same) {
    double sv[kMaxPoly];
    unsigned inside = 0;
    for (int i = 0; i < n; ++i) {
        double s = c0;
#pragma unroll
        for (int j = 0; j < D; ++j) s = fma(g[j], in[i][j], s);
        sv[i] = s;
        inside |= (unsigned)nonneg_d(s) << i;
    }
    const unsigned all = (1u << n) - 1u;
    same = inside == all;
    if (same) return n;
    if (inside == 0) return 0;
    int e0, e1;
    const bool repaired = !one_run(inside, n, e0, e1);
    if (repaired) {
        int j = -1;
        for (int i = 0; i < n; ++i)
            if (!((inside >> i) & 1u) && (j < 0 || sv[i] < sv[j])) j = i;
        inside = keep_outside_run(~inside & all, n, j);
        one_run(inside, n, e0, e1);
    }
    double t[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int i = r == 0 ? e0 : e1;
        const int i1 = i + 1 == n ? 0 : i + 1;
        t[r] = kFastDiv ? div_fast(sv[i], sv[i] - sv[i1]) : div_nr(sv[i], sv[i] - sv[i1]);
    }
    if (repaired) {
        t[0] = clamp01(t[0]);
        t[1] = clamp01(t[1]);
    }
    double X[2][D];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int i = r == 0 ? e0 : e1;
        const double* p = in[i];
        const double* q = in[i + 1 == n ? 0 : i + 1];
#pragma unroll
        for (int j = 0; j < D; ++j) X[r][j] = fma(t[r], q[j] - p[j], p[j]);
    }
    return clip_emit<D>(in, n, inside, e0, X[0], e1, X[1], out);
}

// ------------------------------------------------------------------ moments
// Moment slots: mu[S] (S = axis bit set, 2^D slots) then sq[j][T] = ∫ u_j^2 u^T
// (T a subset of the other axes; 2^(D-1) slots per j).
template <int D>
struct MomentLayout {
    static constexpr int kMu = 1 << D;
    static constexpr int kSqPer = 1 << (D - 1);
    static constexpr int kN = kMu + D * kSqPer;  // 8 (2-D) / 20 (3-D)
};

// Cone triangle (0, q, r) in 2-D: Dv = 2*signed area.  ∫_T = Dv / (2+deg)! * sum.
template <typename R>
__device__ __forceinline__ void cone_accum2(const R* q, const R* r, R Dv, R* acc) {
    R s0 = q[0] + r[0], s1 = q[1] + r[1];
    R P00 = q[0] * q[0] + r[0] * r[0];
    R P11 = q[1] * q[1] + r[1] * r[1];
    R P01 = q[0] * q[1] + r[0] * r[1];
    R Q001 = q[0] * q[0] * q[1] + r[0] * r[0] * r[1];
    R Q110 = q[1] * q[1] * q[0] + r[1] * r[1] * r[0];
    acc[0] += Dv;
    acc[1] += Dv * s0;
    acc[2] += Dv * s1;
    acc[3] += Dv * (s0 * s1 + P01);
    acc[4] += Dv * (s0 * s0 + P00);                                          // u0^2
    acc[5] += Dv * (s0 * s0 * s1 + R(2) * s0 * P01 + s1 * P00 + R(2) * Q001);  // u0^2 u1
    acc[6] += Dv * (s1 * s1 + P11);                                          // u1^2
    acc[7] += Dv * (s1 * s1 * s0 + R(2) * s1 * P01 + s0 * P11 + R(2) * Q110);  // u1^2 u0
}

template <typename R>
__device__ __forceinline__ void finish_moments2(R* acc) {
    acc[0] *= R(1.0 / 2.0);
    acc[1] *= R(1.0 / 6.0);
    acc[2] *= R(1.0 / 6.0);
    acc[3] *= R(1.0 / 24.0);
    acc[4] *= R(1.0 / 24.0);
    acc[6] *= R(1.0 / 24.0);
    acc[5] *= R(1.0 / 120.0);
    acc[7] *= R(1.0 / 120.0);
}

// Cone tetrahedron (0, p, q, r) in 3-D: Dv = 6*signed volume.  ∫_T = Dv/(3+deg)! * sum.
template <typename R>
__device__ __forceinline__ R det3(const R* p, const R* q, const R* r) {
    return p[0] * (q[1] * r[2] - q[2] * r[1]) + p[1] * (q[2] * r[0] - q[0] * r[2]) + p[2] * (q[0] * r[1] - q[1] * r[0]);
}

// The same determinant in double-float arithmetic (FP32 instructions only): the
// intersection volume of the mixed form keeps FP64-level accuracy without
// issuing to the narrow FP64 unit.
__device__ __forceinline__ DF df_det3(const DF* p, const DF* q, const DF* r) {
    const DF c0 = df_add(df_mul(q[1], r[2]), df_neg(df_mul(q[2], r[1])));
    const DF c1 = df_add(df_mul(q[2], r[0]), df_neg(df_mul(q[0], r[2])));
    const DF c2 = df_add(df_mul(q[0], r[1]), df_neg(df_mul(q[1], r[0])));
    return df_add(df_add(df_mul(p[0], c0), df_mul(p[1], c1)), df_mul(p[2], c2));
}
__device__ __forceinline__ DF df_det2(const DF* q, const DF* r) {
    return df_add(df_mul(q[0], r[1]), df_neg(df_mul(q[1], r[0])));
}

// Moments of the tetrahedron (apex, p, q, r): the power sums run over all four
// vertices; with ap == nullptr the apex is the origin and drops out, else it is
// the point ap[0..2].
template <typename R>
__device__ __forceinline__ void cone_accum3(const R* p, const R* q, const R* r, R Dv, R* acc,
                                            const R* ap = nullptr) {
    R s[3], P[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) s[k] = p[k] + q[k] + r[k] + (ap ? ap[k] : R(0));
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = k; l < 3; ++l) {
            P[k][l] = p[k] * p[l] + q[k] * q[l] + r[k] * r[l] + (ap ? ap[k] * ap[l] : R(0));
            P[l][k] = P[k][l];
        }
    R Q012 = p[0] * p[1] * p[2] + q[0] * q[1] * q[2] + r[0] * r[1] * r[2] + (ap ? ap[0] * ap[1] * ap[2] : R(0));
    acc[0] += Dv;
    acc[1] += Dv * s[0];
    acc[2] += Dv * s[1];
    acc[4] += Dv * s[2];
    acc[3] += Dv * (s[0] * s[1] + P[0][1]);
    acc[5] += Dv * (s[0] * s[2] + P[0][2]);
    acc[6] += Dv * (s[1] * s[2] + P[1][2]);
    acc[7] += Dv * (s[0] * s[1] * s[2] + s[0] * P[1][2] + s[1] * P[0][2] + s[2] * P[0][1] + R(2) * Q012);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int a = (j + 1) % 3, b = (j + 2) % 3;
        R pj2 = p[j] * p[j], qj2 = q[j] * q[j], rj2 = r[j] * r[j];
        const R aj2 = ap ? ap[j] * ap[j] : R(0);
        R Qjja = pj2 * p[a] + qj2 * q[a] + rj2 * r[a] + (ap ? aj2 * ap[a] : R(0));
        R Qjjb = pj2 * p[b] + qj2 * q[b] + rj2 * r[b] + (ap ? aj2 * ap[b] : R(0));
        R Rjjab = pj2 * p[a] * p[b] + qj2 * q[a] * q[b] + rj2 * r[a] * r[b] + (ap ? aj2 * ap[a] * ap[b] : R(0));
        R sj = s[j], sa = s[a], sb = s[b];
        acc[8 + 4 * j + 0] += Dv * (sj * sj + P[j][j]);
        acc[8 + 4 * j + 1] += Dv * (sj * sj * sa + R(2) * sj * P[j][a] + sa * P[j][j] + R(2) * Qjja);
        acc[8 + 4 * j + 2] += Dv * (sj * sj * sb + R(2) * sj * P[j][b] + sb * P[j][j] + R(2) * Qjjb);
        R f4 = sj * sj * sa * sb + P[j][j] * sa * sb + R(2) * sj * (P[j][a] * sb + P[j][b] * sa) +
               P[a][b] * sj * sj + P[j][j] * P[a][b] + R(2) * P[j][a] * P[j][b] +
               R(2) * (Qjja * sb + Qjjb * sa) + R(4) * Q012 * sj + R(6) * Rjjab;
        acc[8 + 4 * j + 3] += Dv * f4;
    }
}

template <typename R>
__device__ __forceinline__ void finish_moments3(R* acc) {
    acc[0] *= R(1.0 / 6.0);
    acc[1] *= R(1.0 / 24.0);
    acc[2] *= R(1.0 / 24.0);
    acc[4] *= R(1.0 / 24.0);
    acc[3] *= R(1.0 / 120.0);
    acc[5] *= R(1.0 / 120.0);
    acc[6] *= R(1.0 / 120.0);
    acc[7] *= R(1.0 / 720.0);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        acc[8 + 4 * j + 0] *= R(1.0 / 120.0);
        acc[8 + 4 * j + 1] *= R(1.0 / 720.0);
        acc[8 + 4 * j + 2] *= R(1.0 / 720.0);
        acc[8 + 4 * j + 3] *= R(1.0 / 5040.0);
    }
}

// ∫ u_j u^S from the moment slots.
template <int D, typename R>
__device__ __forceinline__ R moment_nu(const R* acc, int j, int S) {
    if ((S >> j) & 1) {
        int rest = S & ~(1 << j);
        int o1 = (j + 1) % D;
        int t = (rest >> o1) & 1;
        if (D == 3) t |= ((rest >> ((j + 2) % 3)) & 1) << 1;
        return acc[(1 << D) + j * (1 << (D - 1)) + t];
    }
    return acc[S | (1 << j)];
}

// Frame of the FP32 moments of the mixed 3-D form: they are taken about a point
// c near the middle of E ∩ C (c given in apex coordinates, a float), not about
// the apex, so that they carry no large offset that the contraction with
// lambda_a psi_b would cancel (the apex sits on the crossed cell planes and can
// lie a few element sizes from the element).  The apex becomes the fourth
// vertex -c of every cone tetrahedron.
struct ShiftFrame {
    float c[3];   // the point, apex coordinates
    float a[3];   // the apex in the frame: -c
};

// Fan a polygon given in apex coordinates (apex at the origin) into cone
// simplices and accumulate their moments.  2-D: cone triangles (0, v_i, v_i+1);
// 3-D: cone tetrahedra (0, v_0, v_i, v_i+1).  With R = float the cone volumes
// come from double-float determinants of the FP64 vertices (split into float
// pairs by integer instructions) and their sum is kept in *vol_df; the other
// moments take the vertices relative to the frame's point (3-D; in 2-D the
// apex is a vertex of the polygon itself).
template <int D, typename R>
__device__ __forceinline__ void accum_polygon(const double (*poly)[D], int n, R* acc, DF* vol_df,
                                              const ShiftFrame* fr = nullptr) {
    constexpr bool kDF = sizeof(R) == 4;
    if constexpr (D == 2) {
        R q[2], r[2];
        DF qd[2], rd[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if constexpr (kDF) {
                qd[k] = df_split_int(poly[0][k]);
                q[k] = qd[k].hi;
            } else {
                q[k] = to_r<R>(poly[0][k]);
            }
        }
        for (int i = 0; i < n; ++i) {
            const int j = i + 1 == n ? 0 : i + 1;
            R Dv;
            if constexpr (kDF) {
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    rd[k] = df_split_int(poly[j][k]);
                    r[k] = rd[k].hi;
                }
                const DF dv = df_det2(qd, rd);
                *vol_df = df_add(*vol_df, dv);
                Dv = __fadd_rn(dv.hi, dv.lo);
            } else {
                r[0] = to_r<R>(poly[j][0]);
                r[1] = to_r<R>(poly[j][1]);
                Dv = q[0] * r[1] - q[1] * r[0];
            }
            cone_accum2<R>(q, r, Dv, acc);
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                q[k] = r[k];
                if constexpr (kDF) qd[k] = rd[k];
            }
        }
    } else {
        if (n < 3) return;
        R p[3], q[3], r[3];
        DF pd[3], qd[3], rd[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if constexpr (kDF) {
                pd[k] = df_split_int(poly[0][k]);
                qd[k] = df_split_int(poly[1][k]);
                p[k] = __fadd_rn(__fsub_rn(pd[k].hi, fr->c[k]), pd[k].lo);
                q[k] = __fadd_rn(__fsub_rn(qd[k].hi, fr->c[k]), qd[k].lo);
            } else {
                p[k] = to_r<R>(poly[0][k]);
                q[k] = to_r<R>(poly[1][k]);
            }
        }
        for (int i = 1; i + 1 < n; ++i) {
            R Dv;
            if constexpr (kDF) {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    rd[k] = df_split_int(poly[i + 1][k]);
                    r[k] = __fadd_rn(__fsub_rn(rd[k].hi, fr->c[k]), rd[k].lo);
                }
                const DF dv = df_det3(pd, qd, rd);
                *vol_df = df_add(*vol_df, dv);
                Dv = __fadd_rn(dv.hi, dv.lo);
                cone_accum3<R>(p, q, r, Dv, acc, reinterpret_cast<const R*>(fr->a));
            } else {
#pragma unroll
                for (int k = 0; k < 3; ++k) r[k] = to_r<R>(poly[i + 1][k]);
                Dv = det3<R>(p, q, r);
                cone_accum3<R>(p, q, r, Dv, acc);
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                q[k] = r[k];
                if constexpr (kDF) qd[k] = rd[k];
            }
        }
    }
}

// Barycentric coordinates of an element in cell-local coordinates t = (x - c)/h:
// lambda_a(t) = c_a + g[a] . t, with g independent of the cell.  Edges
// (X_i - X_0) / h, adjugate over determinant.  Returns false for a zero volume.
template <int D>
__device__ __forceinline__ bool elem_gradients(const double (&X)[D + 1][D], const double* inv_h,
                                               double (&g)[D + 1][D], bool& positive) {
    double e[D][D];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int k = 0; k < D; ++k) e[i][k] = (X[i + 1][k] - X[0][k]) * inv_h[k];
    double det;
    if constexpr (D == 2) {
        det = e[0][0] * e[1][1] - e[0][1] * e[1][0];
        if (det == 0.0) return false;
        const double id = div_nr(1.0, det);
        g[1][0] = e[1][1] * id;
        g[1][1] = -e[1][0] * id;
        g[2][0] = -e[0][1] * id;
        g[2][1] = e[0][0] * id;
    } else {
        const double c0[3] = {e[1][1] * e[2][2] - e[1][2] * e[2][1], e[1][2] * e[2][0] - e[1][0] * e[2][2],
                              e[1][0] * e[2][1] - e[1][1] * e[2][0]};
        det = e[0][0] * c0[0] + e[0][1] * c0[1] + e[0][2] * c0[2];
        if (det == 0.0) return false;
        const double id = div_nr(1.0, det);
        const double c1[3] = {e[2][1] * e[0][2] - e[2][2] * e[0][1], e[2][2] * e[0][0] - e[2][0] * e[0][2],
                              e[2][0] * e[0][1] - e[2][1] * e[0][0]};
        const double c2[3] = {e[0][1] * e[1][2] - e[0][2] * e[1][1], e[0][2] * e[1][0] - e[0][0] * e[1][2],
                              e[0][0] * e[1][1] - e[0][1] * e[1][0]};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            g[1][k] = c0[k] * id;
            g[2][k] = c1[k] * id;
            g[3][k] = c2[k] * id;
        }
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
        double s = 0.0;
#pragma unroll
        for (int a = 1; a <= D; ++a) s += g[a][k];
        g[0][k] = -s;
    }
    positive = det > 0.0;
    return true;
}

// Classification of a pair from the element's vertices in cell-local
// coordinates: returns false if the overlap has zero measure; sets the masks of
// crossed lower / upper cell planes and of vertices inside the closed cell.
template <int D>
__device__ __forceinline__ bool classify_pair(const double (&T)[D + 1][D], long long (&kmin)[D], long long (&kmax)[D],
                                              int& lower_mask, int& upper_mask, int& inside_mask) {
    constexpr int NA = D + 1;
    constexpr long long K1 = 0x3ff0000000000000LL;  // order key of 1.0 (key of +0.0 is 0)
    lower_mask = upper_mask = 0;
    inside_mask = (1 << NA) - 1;
    bool live = true;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        kmin[k] = LLONG_MAX;
        kmax[k] = LLONG_MIN;
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            const long long kk = order_key(T[a][k]);
            kmin[k] = min(kmin[k], kk);
            kmax[k] = max(kmax[k], kk);
            if (kk < 0 || kk > K1) inside_mask &= ~(1 << a);
        }
        if (kmax[k] <= 0 || kmin[k] >= K1) live = false;
        if (kmin[k] < 0) lower_mask |= 1 << k;
        if (kmax[k] > K1) upper_mask |= 1 << k;
    }
    return live;
}

// Scheduling class of a pair (pairs of one class run the same plane lists):
// 0 = no overlap, else 1 + 2 * (the crossed lower and upper cell planes as a
// 2d-bit mask) + (a vertex inside the cell); at most 2^(2d+1) + 1 classes.
template <int D>
__device__ __forceinline__ int pair_class(const double (&T)[D + 1][D]) {
    long long kmin[D], kmax[D];
    int lo, up, in;
    if (!classify_pair<D>(T, kmin, kmax, lo, up, in)) return 0;
    return 1 + 2 * (lo | (up << D)) + (in ? 1 : 0);
}

// Zero block of a pair without overlap, in 32-byte stores.
template <int D>
__device__ __forceinline__ void store_zero_block(double* block) {
#pragma unroll
    for (int i = 0; i < (D + 1) << D; i += 4)
        reinterpret_cast<double4_32a*>(block)[i / 4] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
}

// Clip + integrate one pair.  T: element vertices in cell-local coordinates;
// g, positive: from elem_gradients; scale = volume of the cell.  Writes the
// (d+1)*2^d block straight to `block` (32-byte aligned, row-major by element
// vertex) and the intersection volume to *vol.
template <int D, typename R>
__device__ void pair_integrals(const double (&T)[D + 1][D], const double (&g)[D + 1][D], bool positive,
                               double scale, double* block, double* vol, double (*poly)[D]) {
    constexpr int NB = 1 << D;
    constexpr int NA = D + 1;
    using L = MomentLayout<D>;
    constexpr long long K1 = 0x3ff0000000000000LL;  // order key of 1.0 (key of +0.0 is 0)
    // the mixed precision form takes the crossing parameters to about 2^-45
    // (div_fast), the FP64 form to two ulps (div_nr)
    constexpr bool kFast = sizeof(R) == 4;
    long long kmin[D], kmax[D];
    int lower_mask, upper_mask, inside_mask;
    if (!classify_pair<D>(T, kmin, kmax, lower_mask, upper_mask, inside_mask)) {  // no overlap of positive measure
        store_zero_block<D>(block);
        *vol = 0.0;
        return;
    }
    // 3-D: an element vertex is the apex only when the element crosses no cell
    // plane; otherwise the apex sits on the crossed planes (fewer faces to clip)
    const int apex_v = (inside_mask && (D == 2 || (lower_mask | upper_mask) == 0)) ? __ffs(inside_mask) - 1 : -1;
    double A[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        if (apex_v >= 0) {
            A[k] = T[apex_v][k];
        } else if (D == 3 && ((lower_mask >> k) & 1)) {
            A[k] = 0.0;  // on the crossed plane: its cell face has a zero-volume cone
        } else if (D == 3 && ((upper_mask >> k) & 1)) {
            A[k] = 1.0;
        } else {
            // any point of the overlap serves: a float midpoint, no FP64 arithmetic
            const float lo = d2f_int(from_order_key(max(kmin[k], 0LL)));
            const float hi = d2f_int(from_order_key(min(kmax[k], K1)));
            A[k] = f2d_int(0.5f * (lo + hi));
        }
    }
    // lambda_a at the apex: c'_a = -g_a . (T_0 - A) for a >= 1, c'_0 = 1 - sum
    double cA[NA];
    {
        double u0[D];
#pragma unroll
        for (int k = 0; k < D; ++k) u0[k] = T[0][k] - A[k];
        double csum = 0.0;
#pragma unroll
        for (int a = 1; a < NA; ++a) {
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) v = fma(-g[a][k], u0[k], v);
            cA[a] = v;
            csum += v;
        }
        cA[0] = 1.0 - csum;
    }
    R acc[L::kN];
#pragma unroll
    for (int i = 0; i < L::kN; ++i) acc[i] = R(0);
    DF vol_df{0.0f, 0.0f};  // D! x |E ∩ C| in double-float (mixed form)
    // mixed 3-D form: the frame of the FP32 moments (a point near the middle of
    // E ∩ C, apex coordinates) and lambda_a there in double-float
    constexpr bool kShift = sizeof(R) == 4 && D == 3;
    ShiftFrame fr{};
    if constexpr (kShift) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float ck = 0.0f;  // uncrossed axis: the apex is already at the middle of the overlap
            if (apex_v >= 0)  // element inside the cell: its centroid
                ck = __fsub_rn(0.25f * (d2f_int(T[0][k]) + d2f_int(T[1][k]) + d2f_int(T[2][k]) + d2f_int(T[3][k])),
                               d2f_int(A[k]));
            else if ((lower_mask >> k) & 1)  // apex at t_k = 0, E ∩ C within [0, min(t_max, 1)]
                ck = 0.5f * d2f_int(from_order_key(min(kmax[k], K1)));
            else if ((upper_mask >> k) & 1)  // apex at t_k = 1, E ∩ C within [max(t_min, 0), 1]
                ck = 0.5f * __fsub_rn(d2f_int(from_order_key(max(kmin[k], 0LL))), 1.0f);
            fr.c[k] = ck;
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) fr.a[k] = -fr.c[k];
    }
    // the two polygon buffers (2 * kMaxPoly vertices), owned by the caller
    double (*bufA)[D] = poly;
    double (*bufB)[D] = poly + kMaxPoly;
    if constexpr (D == 2) {
        // P = triangle clipped by the crossed cell lines (counter-clockwise), then
        // re-centred on its first vertex, which becomes the apex.
        int n = 3;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int v = positive ? i : 2 - i;
#pragma unroll
            for (int k = 0; k < D; ++k) bufA[i][k] = T[v][k];
        }
        double (*cur)[D] = bufA;
        double (*nxt)[D] = bufB;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            bool same;
            if ((lower_mask >> k) & 1) { n = clip_axis<D, kFast>(cur, n, nxt, k, 0.0, false, same); if (!same) { double (*t)[D] = cur; cur = nxt; nxt = t; } }
            if ((upper_mask >> k) & 1) { n = clip_axis<D, kFast>(cur, n, nxt, k, 1.0, true, same); if (!same) { double (*t)[D] = cur; cur = nxt; nxt = t; } }
        }
        if (n >= 3) {
            double P0[D];
#pragma unroll
            for (int k = 0; k < D; ++k) P0[k] = cur[0][k];
            for (int i = 0; i < n; ++i)
#pragma unroll
                for (int k = 0; k < D; ++k) cur[i][k] -= P0[k];
            // lambda at the new apex
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                double v = cA[a];
#pragma unroll
                for (int k = 0; k < D; ++k) v = fma(g[a][k], P0[k] - A[k], v);
                cA[a] = v;
            }
#pragma unroll
            for (int k = 0; k < D; ++k) A[k] = P0[k];
            accum_polygon<D, R>(cur, n, acc, &vol_df);
        }
        finish_moments2<R>(acc);
    } else {
        // apex coordinates u = t - A: element vertices, cell planes
        double U[NA][3];
#pragma unroll
        for (int a = 0; a < NA; ++a)
#pragma unroll
            for (int k = 0; k < 3; ++k) U[a][k] = T[a][k] - A[k];
        double clo[3], chi[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            clo[k] = -A[k];
            chi[k] = 1.0 - A[k];
        }
        // crossed cell planes as a compact list (its length is the same for every
        // pair of a scheduling class, so the loops below stay converged)
        int plane_k[6], plane_up[6];
        double plane_c[6];
        int n_planes = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if ((lower_mask >> k) & 1) { plane_k[n_planes] = k; plane_up[n_planes] = 0; plane_c[n_planes] = clo[k]; ++n_planes; }
            if ((upper_mask >> k) & 1) { plane_k[n_planes] = k; plane_up[n_planes] = 1; plane_c[n_planes] = chi[k]; ++n_planes; }
        }
        // The polygons of the boundary of E ∩ C in one loop, so that the clipping and
        // integration code is inlined once: the element faces (face opposite vertex
        // f, outward for a positive element; with an element vertex as apex only
        // the face opposite it has a cone) clipped to the crossed cell planes, then
        // the cell faces the element crosses clipped to the element (a face whose
        // plane holds the apex spans a cone of zero volume and is skipped).
        const int faces[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};
        const int n_faces = apex_v >= 0 ? 1 : 4;
#pragma unroll 1
        for (int jj = 0; jj < n_faces + n_planes; ++jj) {
            double (*cur)[D] = bufA;
            double (*nxt)[D] = bufB;
            int n;
            if (jj < n_faces) {
                const int f = apex_v >= 0 ? apex_v : jj;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const int v = faces[f][positive ? i : 2 - i];
#pragma unroll
                    for (int k = 0; k < 3; ++k) bufA[i][k] = U[v][k];
                }
                n = 3;
#pragma unroll 1
                for (int jp = 0; jp < n_planes; ++jp) {
                    bool same;
                    n = clip_axis<D, kFast>(cur, n, nxt, plane_k[jp], plane_c[jp], plane_up[jp] != 0, same);
                    if (!same) { double (*t)[D] = cur; cur = nxt; nxt = t; }
                }
            } else {
                const int jp = jj - n_faces;
                if ((__double_as_longlong(plane_c[jp]) << 1) == 0) continue;  // c = +-0: the apex's plane
                const int k = plane_k[jp];
                const int side = plane_up[jp];
                const int j1 = (k + 1) % 3, j2 = (k + 2) % 3;
                const double ck = plane_c[jp];
                const double a1[4] = {clo[j1], chi[j1], chi[j1], clo[j1]};
                const double a2[4] = {clo[j2], clo[j2], chi[j2], chi[j2]};
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int sidx = side == 1 ? v : 3 - v;  // outward: +e_k on t_k = 1, -e_k on t_k = 0
                    bufA[v][k] = ck;
                    bufA[v][j1] = a1[sidx];
                    bufA[v][j2] = a2[sidx];
                }
                n = 4;
#pragma unroll 1
                for (int a = 0; a < NA; ++a) {
                    // the plane's coefficients by selects: registers, not a local array
                    const double ca = a == 0 ? cA[0] : a == 1 ? cA[1] : a == 2 ? cA[2] : cA[3];
                    double ga[3];
#pragma unroll
                    for (int k = 0; k < 3; ++k) ga[k] = a == 0 ? g[0][k] : a == 1 ? g[1][k] : a == 2 ? g[2][k] : g[3][k];
                    bool same;
                    n = clip_plane<D, kFast>(cur, n, nxt, ga, ca, same);
                    if (!same) { double (*t)[D] = cur; cur = nxt; nxt = t; }
                }
            }
            accum_polygon<D, R>(cur, n, acc, &vol_df, &fr);
        }
        finish_moments3<R>(acc);
    }
    // lambda_a = cA[a] + g[a].u and psi_b = prod_k (alpha_bk + sigma_bk u_k) around the apex
    const R scale_r = to_r<R>(scale);
    if constexpr (sizeof(R) == 4) *vol = df_to_double(vol_df) * (scale * (D == 3 ? 1.0 / 6.0 : 0.5));
    else *vol = (double)acc[0] * scale;
    // lambda_a at the origin of the moments: at the apex, or (mixed 3-D form) at
    // the frame's point, in double-float
    R cC[NA];
    if constexpr (kShift) {
        DF c0{1.0f, 0.0f};
#pragma unroll
        for (int a = 1; a < NA; ++a) {
            DF v = df_split_int(cA[a]);
#pragma unroll
            for (int k = 0; k < 3; ++k) v = df_add(v, df_mul(df_split_int(g[a][k]), DF{fr.c[k], 0.0f}));
            cC[a] = __fadd_rn(v.hi, v.lo);
            c0 = df_add(c0, df_neg(v));
        }
        cC[0] = __fadd_rn(c0.hi, c0.lo);
    } else {
#pragma unroll
        for (int a = 0; a < NA; ++a) cC[a] = to_r<R>(cA[a]);
    }
    R W[NB], Wj[NB][D];
    R Ar[D], A1r[D];  // psi_b factors t_k and 1 - t_k at the origin of the moments
#pragma unroll
    for (int k = 0; k < D; ++k) {
        if constexpr (kShift) {
            Ar[k] = __fadd_rn(d2f_int(A[k]), fr.c[k]);
            A1r[k] = __fsub_rn(1.0f, Ar[k]);
        } else {
            Ar[k] = to_r<R>(A[k]);
            A1r[k] = to_r<R>(1.0 - A[k]);
        }
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        R coef[NB];
#pragma unroll
        for (int S = 0; S < NB; ++S) {
            R cf = R(1);
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const bool bk = (b >> k) & 1;
                if ((S >> k) & 1) cf = bk ? cf : -cf;
                else cf *= bk ? Ar[k] : A1r[k];
            }
            coef[S] = cf;
        }
        R w = R(0);
#pragma unroll
        for (int S = 0; S < NB; ++S) w += coef[S] * acc[S];
        W[b] = w;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            R v = R(0);
#pragma unroll
            for (int S = 0; S < NB; ++S) v += coef[S] * moment_nu<D, R>(acc, j, S);
            Wj[b][j] = v;
        }
    }
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const R ca = cC[a];
        R ga[D];
#pragma unroll
        for (int k = 0; k < D; ++k) ga[k] = to_r<R>(g[a][k]);
        double row[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            R v = ca * W[b];
#pragma unroll
            for (int j = 0; j < D; ++j) v += ga[j] * Wj[b][j];
            if constexpr (sizeof(R) == 4) row[b] = f2d_int(v * scale_r);
            else row[b] = (double)v * scale;
        }
#pragma unroll
        for (int b = 0; b < NB; b += 4)
            reinterpret_cast<double4_32a*>(block + a * NB)[b / 4] = make_double4_32a(row[b], row[b + 1], row[b + 2], row[b + 3]);
    }
}

}  // namespace l2x
