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
//    signed simplices (divergence theorem).  A is an element vertex lying in
//    the cell when there is one (then the element faces through it drop out
//    and every cone is non-negative), else the centre of the overlap of the
//    element's bounding box with the cell.
//  * On each cone simplex (0, p, q[, r]) in u = t - A the monomial moments
//    needed for lambda_a psi_b (u^S and u_j u^S, S a subset of the axes) are
//    exact closed forms: for a simplex T and monomial prod_j u_{k_j} of degree
//    q, ∫_T = |T| n!/(n+q)! sum over permutations sigma of S_q of
//    prod over cycles c of sigma of (sum over vertices v of prod_{j in c} v_{k_j}).
//  * Geometry (plane tests, intersection points) is always FP64; the moment
//    arithmetic runs in R = double (FP64 mode) or R = float (mixed mode).
#pragma once

#include "l2x_internal.cuh"

namespace l2x {

constexpr int kMaxPoly = 10;  // triangle + 6 planes -> 9; square + 4 planes -> 8

template <int D>
struct ElemT {
    double T[D + 1][D];   // vertices in cell-local coordinates
};

// Sutherland-Hodgman step against an axis plane: keep v[k] >= c (upper=false)
// or v[k] <= c (upper=true).  Intersection points are put on the plane exactly.
template <int D>
__device__ __forceinline__ int clip_axis(const double (*in)[D], int n, double (*out)[D], int k, double c,
                                         bool upper) {
    int m = 0;
    for (int i = 0; i < n; ++i) {
        const double* p = in[i];
        const double* q = in[i + 1 == n ? 0 : i + 1];
        double sp = upper ? c - p[k] : p[k] - c;
        double sq = upper ? c - q[k] : q[k] - c;
        bool ip = sp >= 0.0, iq = sq >= 0.0;
        if (ip) {
#pragma unroll
            for (int j = 0; j < D; ++j) out[m][j] = p[j];
            ++m;
        }
        if (ip != iq) {
            double t = sp / (sp - sq);
#pragma unroll
            for (int j = 0; j < D; ++j) out[m][j] = fma(t, q[j] - p[j], p[j]);
            out[m][k] = c;
            ++m;
        }
    }
    return m;
}

// Sutherland-Hodgman step against the half-space g.v + c0 >= 0.
template <int D>
__device__ __forceinline__ int clip_plane(const double (*in)[D], int n, double (*out)[D], const double* g,
                                          double c0) {
    int m = 0;
    double sp = c0, s0;
#pragma unroll
    for (int j = 0; j < D; ++j) sp = fma(g[j], in[0][j], sp);
    s0 = sp;
    for (int i = 0; i < n; ++i) {
        const double* p = in[i];
        const double* q = in[i + 1 == n ? 0 : i + 1];
        double sq;
        if (i + 1 == n) {
            sq = s0;
        } else {
            sq = c0;
#pragma unroll
            for (int j = 0; j < D; ++j) sq = fma(g[j], q[j], sq);
        }
        bool ip = sp >= 0.0, iq = sq >= 0.0;
        if (ip) {
#pragma unroll
            for (int j = 0; j < D; ++j) out[m][j] = p[j];
            ++m;
        }
        if (ip != iq) {
            double t = sp / (sp - sq);
#pragma unroll
            for (int j = 0; j < D; ++j) out[m][j] = fma(t, q[j] - p[j], p[j]);
            ++m;
        }
        sp = sq;
    }
    return m;
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

// Cone triangle (0, q, r) in 2-D: D2 = 2*signed area.  ∫_T = D2 / (2+deg)! * sum.
template <typename R>
__device__ __forceinline__ void cone_accum2(const R* q, const R* r, R* acc) {
    R Dv = q[0] * r[1] - q[1] * r[0];
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

// Cone tetrahedron (0, p, q, r) in 3-D: D6 = 6*signed volume.  ∫_T = D6/(3+deg)! * sum.
template <typename R>
__device__ __forceinline__ void cone_accum3(const R* p, const R* q, const R* r, R* acc) {
    R Dv = p[0] * (q[1] * r[2] - q[2] * r[1]) + p[1] * (q[2] * r[0] - q[0] * r[2]) +
           p[2] * (q[0] * r[1] - q[1] * r[0]);
    R s[3], P[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) s[k] = p[k] + q[k] + r[k];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int l = k; l < 3; ++l) {
            P[k][l] = p[k] * p[l] + q[k] * q[l] + r[k] * r[l];
            P[l][k] = P[k][l];
        }
    R Q012 = p[0] * p[1] * p[2] + q[0] * q[1] * q[2] + r[0] * r[1] * r[2];
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
        R Qjja = pj2 * p[a] + qj2 * q[a] + rj2 * r[a];
        R Qjjb = pj2 * p[b] + qj2 * q[b] + rj2 * r[b];
        R Rjjab = pj2 * p[a] * p[b] + qj2 * q[a] * q[b] + rj2 * r[a] * r[b];
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

// Fan a polygon (in t-space) into cone simplices with apex A and accumulate.
template <int D, typename R>
__device__ __forceinline__ void accum_polygon(const double (*poly)[D], int n, const double* A, R* acc) {
    if constexpr (D == 2) {
        // 2-D: the polygon is P itself; apex = its vertex 0 (A is ignored).
        R q[2], r[2];
        for (int i = 1; i + 1 < n; ++i) {
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                q[k] = (R)(poly[i][k] - poly[0][k]);
                r[k] = (R)(poly[i + 1][k] - poly[0][k]);
            }
            cone_accum2<R>(q, r, acc);
        }
    } else {
        if (n < 3) return;
        R p[3], q[3], r[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) p[k] = (R)(poly[0][k] - A[k]);
        for (int i = 1; i + 1 < n; ++i) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                q[k] = (R)(poly[i][k] - A[k]);
                r[k] = (R)(poly[i + 1][k] - A[k]);
            }
            cone_accum3<R>(p, q, r, acc);
        }
    }
}

// Clip + integrate one pair.  T: element vertices in cell-local coordinates.
// scale = h0*h1(*h2) (volume of the cell).  Writes (d+1)*2^d block entries and
// the intersection volume.  Returns false if the element is degenerate.
template <int D, typename R>
__device__ bool pair_integrals(const double (&T)[D + 1][D], double scale, double* block, double* vol) {
    constexpr int NB = 1 << D;
    constexpr int NA = D + 1;
    using L = MomentLayout<D>;
    // crossing mask and bounds
    double mn[D], mx[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        mn[k] = T[0][k];
        mx[k] = T[0][k];
#pragma unroll
        for (int a = 1; a < NA; ++a) {
            mn[k] = fmin(mn[k], T[a][k]);
            mx[k] = fmax(mx[k], T[a][k]);
        }
    }
    *vol = 0.0;
#pragma unroll
    for (int i = 0; i < NA * NB; ++i) block[i] = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k)
        if (mx[k] <= 0.0 || mn[k] >= 1.0) return true;  // no overlap of positive measure
    int lower_mask = 0, upper_mask = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        if (mn[k] < 0.0) lower_mask |= 1 << k;
        if (mx[k] > 1.0) upper_mask |= 1 << k;
    }
    // barycentric coordinates in t-space: lambda_a(t) = c[a] + g[a] . t
    double g[NA][D], c[NA];
    double det;
    if constexpr (D == 2) {
        double e1x = T[1][0] - T[0][0], e1y = T[1][1] - T[0][1];
        double e2x = T[2][0] - T[0][0], e2y = T[2][1] - T[0][1];
        det = e1x * e2y - e1y * e2x;
        if (det == 0.0) return false;
        double id = 1.0 / det;
        g[1][0] = e2y * id; g[1][1] = -e2x * id;
        g[2][0] = -e1y * id; g[2][1] = e1x * id;
    } else {
        double e[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k) e[i][k] = T[i + 1][k] - T[0][k];
        // rows of the inverse edge matrix: (e1 x e2, e2 x e0, e0 x e1) / det
        double c0[3] = {e[1][1] * e[2][2] - e[1][2] * e[2][1], e[1][2] * e[2][0] - e[1][0] * e[2][2],
                        e[1][0] * e[2][1] - e[1][1] * e[2][0]};
        det = e[0][0] * c0[0] + e[0][1] * c0[1] + e[0][2] * c0[2];
        if (det == 0.0) return false;
        double id = 1.0 / det;
        double c1[3] = {e[2][1] * e[0][2] - e[2][2] * e[0][1], e[2][2] * e[0][0] - e[2][0] * e[0][2],
                        e[2][0] * e[0][1] - e[2][1] * e[0][0]};
        double c2[3] = {e[0][1] * e[1][2] - e[0][2] * e[1][1], e[0][2] * e[1][0] - e[0][0] * e[1][2],
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
        double sgk = 0.0;
#pragma unroll
        for (int a = 1; a < NA; ++a) sgk += g[a][k];
        g[0][k] = -sgk;
    }
    {
        double csum = 0.0;
#pragma unroll
        for (int a = 1; a < NA; ++a) {
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) v = fma(-g[a][k], T[0][k], v);
            c[a] = v;
            csum += v;
        }
        c[0] = 1.0 - csum;
    }
    // apex: an element vertex inside the closed cell, else the centre of bbox ∩ cell
    int apex_v = -1;
#pragma unroll
    for (int a = NA - 1; a >= 0; --a) {
        bool in = true;
#pragma unroll
        for (int k = 0; k < D; ++k) in = in && T[a][k] >= 0.0 && T[a][k] <= 1.0;
        if (in) apex_v = a;
    }
    double A[D];
#pragma unroll
    for (int k = 0; k < D; ++k)
        A[k] = apex_v >= 0 ? T[apex_v][k] : 0.5 * (fmax(mn[k], 0.0) + fmin(mx[k], 1.0));

    R acc[L::kN];
#pragma unroll
    for (int i = 0; i < L::kN; ++i) acc[i] = R(0);

    double bufA[kMaxPoly][D], bufB[kMaxPoly][D];
    const bool positive = det > 0.0;
    if constexpr (D == 2) {
        // P = triangle clipped by the crossed cell lines; oriented counter-clockwise
        int n = 3;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            int v = positive ? i : 2 - i;
#pragma unroll
            for (int k = 0; k < D; ++k) bufA[i][k] = T[v][k];
        }
        double (*cur)[D] = bufA;
        double (*nxt)[D] = bufB;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            if ((lower_mask >> k) & 1) { n = clip_axis<D>(cur, n, nxt, k, 0.0, false); double (*t)[D] = cur; cur = nxt; nxt = t; }
            if ((upper_mask >> k) & 1) { n = clip_axis<D>(cur, n, nxt, k, 1.0, true); double (*t)[D] = cur; cur = nxt; nxt = t; }
        }
        if (n >= 3) {
            // 2-D apex: vertex 0 of P (the fan below cones every triangle to it)
#pragma unroll
            for (int k = 0; k < D; ++k) A[k] = cur[0][k];
            accum_polygon<D, R>(cur, n, A, acc);
        }
        finish_moments2<R>(acc);
    } else {
        // element faces: face opposite vertex f, outward for a positive element
        const int faces[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};
#pragma unroll 1
        for (int f = 0; f < 4; ++f) {
            if (apex_v >= 0 && apex_v != f) continue;  // face contains the apex: zero cone
            int n = 3;
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                int v = faces[f][positive ? i : 2 - i];
#pragma unroll
                for (int k = 0; k < D; ++k) bufA[i][k] = T[v][k];
            }
            double (*cur)[D] = bufA;
            double (*nxt)[D] = bufB;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                if (n > 0 && ((lower_mask >> k) & 1)) { n = clip_axis<D>(cur, n, nxt, k, 0.0, false); double (*t)[D] = cur; cur = nxt; nxt = t; }
                if (n > 0 && ((upper_mask >> k) & 1)) { n = clip_axis<D>(cur, n, nxt, k, 1.0, true); double (*t)[D] = cur; cur = nxt; nxt = t; }
            }
            accum_polygon<D, R>(cur, n, A, acc);
        }
        // cell faces the element crosses, clipped to the element
#pragma unroll 1
        for (int side = 0; side < 2; ++side) {
            int mask = side == 0 ? lower_mask : upper_mask;
#pragma unroll 1
            for (int k = 0; k < 3; ++k) {
                if (!((mask >> k) & 1)) continue;
                const int i1 = (k + 1) % 3, i2 = (k + 2) % 3;
                const double sq[4][2] = {{0.0, 0.0}, {1.0, 0.0}, {1.0, 1.0}, {0.0, 1.0}};
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    int s = side == 1 ? v : 3 - v;  // outward: +e_k on t_k = 1, -e_k on t_k = 0
                    bufA[v][k] = side == 1 ? 1.0 : 0.0;
                    bufA[v][i1] = sq[s][0];
                    bufA[v][i2] = sq[s][1];
                }
                int n = 4;
                double (*cur)[D] = bufA;
                double (*nxt)[D] = bufB;
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    if (n == 0) break;
                    n = clip_plane<D>(cur, n, nxt, g[a], c[a]);
                    double (*t)[D] = cur; cur = nxt; nxt = t;
                }
                accum_polygon<D, R>(cur, n, A, acc);
            }
        }
        finish_moments3<R>(acc);
    }
    // lambda and psi around the apex: lambda_a = cA[a] + g[a].u, psi_b = prod_k (alpha_bk + sigma_bk u_k)
    *vol = (double)acc[0] * scale;
    R W[NB], Wj[NB][D];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        R coef[NB];
#pragma unroll
        for (int S = 0; S < NB; ++S) {
            R cf = R(1);
#pragma unroll
            for (int k = 0; k < D; ++k) {
                bool bk = (b >> k) & 1;
                if ((S >> k) & 1) cf *= bk ? R(1) : R(-1);
                else cf *= bk ? (R)A[k] : (R)(1.0 - A[k]);
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
        double cA = c[a];
#pragma unroll
        for (int k = 0; k < D; ++k) cA = fma(g[a][k], A[k], cA);
        R ca = (R)cA;
        R ga[D];
#pragma unroll
        for (int k = 0; k < D; ++k) ga[k] = (R)g[a][k];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            R v = ca * W[b];
#pragma unroll
            for (int j = 0; j < D; ++j) v += ga[j] * Wj[b][j];
            block[a * NB + b] = (double)v * scale;
        }
    }
    return true;
}

}  // namespace l2x
