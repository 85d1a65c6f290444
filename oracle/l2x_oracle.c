/*
 * Plain FP64 CPU oracle for the L2-projection transfer between a structured
 * Q1 fluid grid and an unstructured P1 solid mesh (Sec. 2.3, paragraph
 * "Variational Transfer", the mortar integrals B_ij and the assembly steps
 * (I)-(IV) that follow them).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this file.  It shares no code with the
 * CUDA library: it is written as the plain definition, slowly and directly.
 *
 * What it computes, per velocity grid (one Q1 grid per staggered velocity
 * component, Sec. 2.2 "Spatial Discretization"):
 *
 *  (I)   candidate pairs: for element e, every cell whose index range overlaps
 *        the element's bounding box, with the index rule
 *            i_lo = floor((lo - o) / h),  i_hi = ceil((hi - o) / h) - 1
 *        evaluated in IEEE double with one rounded subtraction then one
 *        correctly rounded division (no fused multiply-add, no reciprocal).
 *        Order: element, then cell z, y, x (x fastest).
 *  (II)  the intersection E ∩ C, by splitting the simplex against each of
 *        the 2d half-spaces of the cell into a list of sub-simplices
 *        (intersection points snapped onto the clipping plane);
 *  (III) on every sub-simplex, the integrals of lambda_a * psi_b (lambda_a:
 *        barycentric coordinate a of the element, psi_b: Q1 basis function of
 *        cell corner b) with a collapsed-coordinate tensor Gauss-Legendre rule
 *        (Duffy map of the unit cube onto the simplex; 4 points per direction
 *        in 3-D and 3 in 2-D, exact for the integrand degree d+1 times the
 *        Jacobian), and the volume of E ∩ C.
 *  (IV)  assembly into sparse matrices happens in the Python wrapper.
 *
 * Cell corner b has bits (b0, b1, b2); psi_b = prod_k (b_k ? t_k : 1 - t_k),
 * t_k = (x_k - cell_lo_k) / h_k.  Block layout: block[a * 2^d + b].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EOUTOFGRID 4
#define ORC_EDEGENERATE 5
#define ORC_ENOMEM 2

/* ------------------------------------------------------------------ operation tallies
 * The floating-point operations (additions, subtractions, multiplications,
 * divisions; not fabs, comparisons or copies) that steps (II) and (III) below
 * execute, tallied per thread by category when a function runs, and summed over
 * threads by orc_pair_blocks_counted.  Each tally is the operation count of the
 * statement it stands beside.  Categories:
 *   FRAME   the cell's lower corner and the element vertices relative to it;
 *   CLIP    plane-side values and cut points (step II);
 *   VOLUME  the determinant (volume) of every sub-simplex;
 *   BARY    the barycentric map of the element (per pair here);
 *   QUAD    the Gauss-Legendre evaluation of lambda_a psi_b (step III). */
enum { ORC_OPS_FRAME, ORC_OPS_CLIP, ORC_OPS_VOLUME, ORC_OPS_BARY, ORC_OPS_QUAD, ORC_OPS_N };
static _Thread_local uint64_t t_ops[ORC_OPS_N];
#define TALLY(cat, n) (t_ops[cat] += (uint64_t)(n))

/* ------------------------------------------------------------------ (I) */

static void elem_bbox(int dim, const double* X, const int32_t* E, int64_t e, double* lo, double* hi) {
    for (int k = 0; k < dim; ++k) { lo[k] = INFINITY; hi[k] = -INFINITY; }
    for (int v = 0; v <= dim; ++v) {
        const double* p = X + (int64_t)E[e * (dim + 1) + v] * dim;
        for (int k = 0; k < dim; ++k) {
            if (p[k] < lo[k]) lo[k] = p[k];
            if (p[k] > hi[k]) hi[k] = p[k];
        }
    }
}

/* Number of entries of the increasing array x[0..n) that are <= v (upper) or
 * < v (lower): plain binary search, comparisons only. */
static int64_t count_le(const double* x, int64_t n, double v) {
    int64_t l = 0, r = n;
    while (l < r) {
        int64_t m = (l + r) / 2;
        if (x[m] <= v) l = m + 1; else r = m;
    }
    return l;
}
static int64_t count_lt(const double* x, int64_t n, double v) {
    int64_t l = 0, r = n;
    while (l < r) {
        int64_t m = (l + r) / 2;
        if (x[m] < v) l = m + 1; else r = m;
    }
    return l;
}

/* Cell index range of element e along every axis; returns ORC_EOUTOFGRID if
 * the range leaves the grid.  Cells are half-open [x_i, x_{i+1}): the lowest
 * cell holds the lowest bbox coordinate, the highest cell is the last one that
 * starts below the highest coordinate.  Uniform axes (axis == NULL or
 * axis[k] == NULL): x_i = origin + i h, evaluated as one rounded subtraction and
 * one correctly rounded division; stretched axes: the ncell+1 node coordinates
 * axis[k], searched by comparisons. */
int orc_cell_range(int dim, const int64_t* ncell, const double* origin, const double* h,
                   const double* const* axis, const double* X, const int32_t* E, int64_t e,
                   int64_t* ilo, int64_t* ihi) {
    double lo[3], hi[3];
    elem_bbox(dim, X, E, e, lo, hi);
    for (int k = 0; k < dim; ++k) {
        if (axis && axis[k]) {
            ilo[k] = count_le(axis[k], ncell[k] + 1, lo[k]) - 1;
            ihi[k] = count_lt(axis[k], ncell[k] + 1, hi[k]) - 1;
        } else {
            volatile double dlo = lo[k] - origin[k];
            volatile double dhi = hi[k] - origin[k];
            volatile double qlo = dlo / h[k];
            volatile double qhi = dhi / h[k];
            ilo[k] = (int64_t)floor(qlo);
            ihi[k] = (int64_t)ceil(qhi) - 1;
        }
        if (ihi[k] < ilo[k]) ihi[k] = ilo[k];  /* zero extent along k */
        if (ilo[k] < 0 || ihi[k] >= ncell[k]) return ORC_EOUTOFGRID;
    }
    return ORC_OK;
}

/* counts[e] = number of candidate cells of element e.  Returns 0 or a status;
 * *bad_elem receives the first element that left the grid. */
int orc_count_pairs(int dim, const int64_t* ncell, const double* origin, const double* h,
                    const double* const* axis, int64_t n_elems, const double* X, const int32_t* E,
                    int64_t* counts, int64_t* bad_elem) {
    for (int64_t e = 0; e < n_elems; ++e) {
        int64_t ilo[3], ihi[3];
        if (orc_cell_range(dim, ncell, origin, h, axis, X, E, e, ilo, ihi) != ORC_OK) {
            *bad_elem = e;
            return ORC_EOUTOFGRID;
        }
        int64_t c = 1;
        for (int k = 0; k < dim; ++k) c *= ihi[k] - ilo[k] + 1;
        counts[e] = c;
    }
    return ORC_OK;
}

/* Writes the pair list; offsets[e] = first pair of element e. */
void orc_emit_pairs(int dim, const int64_t* ncell, const double* origin, const double* h,
                    const double* const* axis, int64_t n_elems, const double* X, const int32_t* E,
                    const int64_t* offsets, int32_t* pair_elem, int64_t* pair_cell) {
    for (int64_t e = 0; e < n_elems; ++e) {
        int64_t ilo[3] = {0, 0, 0}, ihi[3] = {0, 0, 0};
        orc_cell_range(dim, ncell, origin, h, axis, X, E, e, ilo, ihi);
        int64_t p = offsets[e];
        int64_t z0 = dim == 3 ? ilo[2] : 0, z1 = dim == 3 ? ihi[2] : 0;
        for (int64_t iz = z0; iz <= z1; ++iz)
            for (int64_t iy = ilo[1]; iy <= ihi[1]; ++iy)
                for (int64_t ix = ilo[0]; ix <= ihi[0]; ++ix) {
                    pair_elem[p] = (int32_t)e;
                    pair_cell[p] = ix + ncell[0] * (iy + ncell[1] * iz);
                    ++p;
                }
    }
}

/* ------------------------------------------------------------------ (II) */

typedef struct { double v[4][3]; } simplex;

typedef struct {
    simplex* s;
    int64_t n, cap;
} slist;

static int slist_push(slist* L, const simplex* s) {
    if (L->n == L->cap) {
        int64_t nc = L->cap ? 2 * L->cap : 16;
        simplex* ns = (simplex*)realloc(L->s, (size_t)nc * sizeof(simplex));
        if (!ns) return ORC_ENOMEM;
        L->s = ns;
        L->cap = nc;
    }
    L->s[L->n++] = *s;
    return ORC_OK;
}

/* signed distance-like value of point p for half-space (axis k, bound c, side):
 * side 0: x_k >= c  ->  x_k - c ;  side 1: x_k <= c  ->  c - x_k.  Inside iff >= 0. */
static double side_value(const double* p, int k, double c, int side) {
    TALLY(ORC_OPS_CLIP, 1);
    return side == 0 ? p[k] - c : c - p[k];
}

/* point on segment p(inside, sp >= 0) -> q(outside, sq < 0) where the plane is met;
 * coordinate k is set to the plane value exactly. */
static void cut_point(int dim, const double* p, const double* q, double sp, double sq, int k,
                      double c, double* r) {
    double t = sp / (sp - sq);
    for (int j = 0; j < dim; ++j) r[j] = p[j] + t * (q[j] - p[j]);
    TALLY(ORC_OPS_CLIP, 2 + 3 * dim);
    r[k] = c;
}

static void set_pt(simplex* s, int i, const double* p, int dim) {
    for (int j = 0; j < dim; ++j) s->v[i][j] = p[j];
}

/* Split one simplex by a half-space; pushes the inside part as simplices. */
static int split_simplex(int dim, const simplex* S, int k, double c, int side, slist* out) {
    int nv = dim + 1;
    double sv[4];
    int in[4], nin = 0, iin[4], iout[4], nout = 0;
    for (int i = 0; i < nv; ++i) {
        sv[i] = side_value(S->v[i], k, c, side);
        in[i] = sv[i] >= 0.0;
        if (in[i]) iin[nin++] = i; else iout[nout++] = i;
    }
    if (nin == 0) return ORC_OK;
    if (nin == nv) return slist_push(out, S);
    simplex T;
    memset(&T, 0, sizeof(T));
    if (dim == 2) {
        if (nin == 1) {
            int a = iin[0], b = iout[0], cc = iout[1];
            double pab[3], pac[3];
            cut_point(2, S->v[a], S->v[b], sv[a], sv[b], k, c, pab);
            cut_point(2, S->v[a], S->v[cc], sv[a], sv[cc], k, c, pac);
            set_pt(&T, 0, S->v[a], 2); set_pt(&T, 1, pab, 2); set_pt(&T, 2, pac, 2);
            return slist_push(out, &T);
        } else { /* nin == 2: quadrilateral a, b, p_bc, p_ac -> two triangles */
            int a = iin[0], b = iin[1], cc = iout[0];
            double pac[3], pbc[3];
            cut_point(2, S->v[a], S->v[cc], sv[a], sv[cc], k, c, pac);
            cut_point(2, S->v[b], S->v[cc], sv[b], sv[cc], k, c, pbc);
            set_pt(&T, 0, S->v[a], 2); set_pt(&T, 1, S->v[b], 2); set_pt(&T, 2, pbc, 2);
            int st = slist_push(out, &T);
            if (st) return st;
            set_pt(&T, 0, S->v[a], 2); set_pt(&T, 1, pbc, 2); set_pt(&T, 2, pac, 2);
            return slist_push(out, &T);
        }
    }
    /* dim == 3 */
    if (nin == 1) {
        int a = iin[0];
        set_pt(&T, 0, S->v[a], 3);
        for (int j = 0; j < 3; ++j) {
            double r[3];
            cut_point(3, S->v[a], S->v[iout[j]], sv[a], sv[iout[j]], k, c, r);
            set_pt(&T, 1 + j, r, 3);
        }
        return slist_push(out, &T);
    }
    /* The inside part is a triangular prism with ends (A,B,C) and (A',B',C'),
     * A-A', B-B', C-C' the lateral edges; it is the union of the three tetrahedra
     * (A,B,C,C'), (A,B,C',B'), (A,B',C',A'). */
    double P[6][3];
    if (nin == 3) { /* ends: the three inside vertices and the cut points toward the outside one */
        int d = iout[0];
        for (int j = 0; j < 3; ++j) {
            int a = iin[j];
            for (int q = 0; q < 3; ++q) P[j][q] = S->v[a][q];
            cut_point(3, S->v[a], S->v[d], sv[a], sv[d], k, c, P[3 + j]);
        }
    } else { /* nin == 2: ends (a, p_ac, p_ad) and (b, p_bc, p_bd) */
        int a = iin[0], b = iin[1], cc = iout[0], d = iout[1];
        for (int q = 0; q < 3; ++q) { P[0][q] = S->v[a][q]; P[3][q] = S->v[b][q]; }
        cut_point(3, S->v[a], S->v[cc], sv[a], sv[cc], k, c, P[1]);
        cut_point(3, S->v[a], S->v[d], sv[a], sv[d], k, c, P[2]);
        cut_point(3, S->v[b], S->v[cc], sv[b], sv[cc], k, c, P[4]);
        cut_point(3, S->v[b], S->v[d], sv[b], sv[d], k, c, P[5]);
    }
    static const int tets[3][4] = {{0, 1, 2, 5}, {0, 1, 5, 4}, {0, 4, 5, 3}};
    for (int t = 0; t < 3; ++t) {
        for (int i = 0; i < 4; ++i) set_pt(&T, i, P[tets[t][i]], 3);
        int st = slist_push(out, &T);
        if (st) return st;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ (III) */

/* Gauss-Legendre nodes/weights on [0,1] for n = 3 and n = 4 (closed forms). */
static void gauss_legendre01(int n, double* x, double* w) {
    if (n == 3) {
        double r = sqrt(3.0 / 5.0);
        double z[3] = {-r, 0.0, r}, wz[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
        for (int i = 0; i < 3; ++i) { x[i] = 0.5 * (1.0 + z[i]); w[i] = 0.5 * wz[i]; }
    } else {
        double r1 = sqrt(3.0 / 7.0 - 2.0 / 7.0 * sqrt(6.0 / 5.0));
        double r2 = sqrt(3.0 / 7.0 + 2.0 / 7.0 * sqrt(6.0 / 5.0));
        double w1 = (18.0 + sqrt(30.0)) / 36.0, w2 = (18.0 - sqrt(30.0)) / 36.0;
        double z[4] = {-r2, -r1, r1, r2}, wz[4] = {w2, w1, w1, w2};
        for (int i = 0; i < 4; ++i) { x[i] = 0.5 * (1.0 + z[i]); w[i] = 0.5 * wz[i]; }
    }
}

/* Inverse of the (d+1)x(d+1) matrix M = [[X_0 .. X_d], [1 .. 1]] by Gauss-Jordan
 * elimination with partial pivoting.  lambda(x) = Minv * (x, 1). */
static int barycentric_map(int dim, double V[4][3], double Minv[4][4]) {
    int n = dim + 1;
    double A[4][8];
    for (int r = 0; r < n; ++r) {
        for (int c = 0; c < n; ++c) A[r][c] = (r < dim) ? V[c][r] : 1.0;
        for (int c = 0; c < n; ++c) A[r][n + c] = (r == c) ? 1.0 : 0.0;
    }
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (A[piv][col] == 0.0) return ORC_EDEGENERATE;
        if (piv != col)
            for (int c = 0; c < 2 * n; ++c) { double t = A[col][c]; A[col][c] = A[piv][c]; A[piv][c] = t; }
        double d = A[col][col];
        for (int c = 0; c < 2 * n; ++c) A[col][c] /= d;
        TALLY(ORC_OPS_BARY, 2 * n);
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            double f = A[r][col];
            for (int c = 0; c < 2 * n; ++c) A[r][c] -= f * A[col][c];
            TALLY(ORC_OPS_BARY, 4 * n);
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) Minv[r][c] = A[r][n + c];
    return ORC_OK;
}

/* Integrates lambda_a * psi_b and 1 over one sub-simplex S. */
static void integrate_simplex(int dim, const simplex* S, double Minv[4][4], const double* clo,
                              const double* h, double* block, double* vol) {
    int nq = dim == 3 ? 4 : 3;
    double gx[4], gw[4];
    gauss_legendre01(nq, gx, gw);
    int nb = 1 << dim, na = dim + 1;
    const double (*p)[3] = S->v;
    double A[3], B[3], C[3];
    for (int j = 0; j < dim; ++j) {
        A[j] = p[1][j] - p[0][j];
        B[j] = p[2][j] - p[1][j];
        C[j] = dim == 3 ? p[3][j] - p[2][j] : 0.0;
    }
    double D;
    if (dim == 2) D = fabs(A[0] * B[1] - A[1] * B[0]);
    else D = fabs(A[0] * (B[1] * C[2] - B[2] * C[1]) - A[1] * (B[0] * C[2] - B[2] * C[0]) +
                  A[2] * (B[0] * C[1] - B[1] * C[0]));
    TALLY(ORC_OPS_VOLUME, dim == 3 ? 9 + 14 : 4 + 3);  /* edge vectors, determinant */
    if (D == 0.0) return;
    int nw = dim == 3 ? nq : 1;
    for (int iu = 0; iu < nq; ++iu)
        for (int iv = 0; iv < nq; ++iv)
            for (int iw = 0; iw < nw; ++iw) {
                double u = gx[iu], v = gx[iv], w = dim == 3 ? gx[iw] : 0.0;
                double wt = gw[iu] * gw[iv] * (dim == 3 ? gw[iw] : 1.0);
                double jac = dim == 3 ? u * u * v * D : u * D;
                /* per point: wt 2, jac 3 (2-D: 1), x 6 per axis, lambda 2*dim per
                 * vertex, t 2 per axis, f 1, vol 1, psi dim products per corner
                 * plus one 1-t per zero bit (dim*nb/2 over all corners), and
                 * 3 per block entry */
                TALLY(ORC_OPS_QUAD, 2 + (dim == 3 ? 3 : 1) + 6 * dim + na * 2 * dim + 2 * dim + 2 +
                                        nb * dim + nb * dim / 2 + 3 * na * nb);
                double x[3];
                for (int j = 0; j < dim; ++j) x[j] = p[0][j] + u * (A[j] + v * (B[j] + w * C[j]));
                double lam[4];
                for (int a = 0; a < na; ++a) {
                    double s = Minv[a][dim];
                    for (int j = 0; j < dim; ++j) s += Minv[a][j] * x[j];
                    lam[a] = s;
                }
                double t[3];
                for (int j = 0; j < dim; ++j) t[j] = (x[j] - clo[j]) / h[j];
                double f = wt * jac;
                *vol += f;
                for (int b = 0; b < nb; ++b) {
                    double psi = 1.0;
                    for (int j = 0; j < dim; ++j) psi *= ((b >> j) & 1) ? t[j] : 1.0 - t[j];
                    for (int a = 0; a < na; ++a) block[a * nb + b] += f * lam[a] * psi;
                }
            }
}

/* Block of one (element, cell) pair: clip (II) then integrate (III).
 * Everything is done in coordinates relative to the cell's lower corner, so that
 * the cell is [0, h_0] x [0, h_1] (x [0, h_2]) and no digits are lost to the
 * absolute position of the pair. */
static int pair_block(int dim, const int64_t* ncell, const double* origin, const double* h_uniform,
                      const double* const* axis, const double* X, const int32_t* E, int64_t e,
                      int64_t cell, double* block, double* vol, slist* L0, slist* L1) {
    int na = dim + 1, nb = 1 << dim;
    for (int i = 0; i < na * nb; ++i) block[i] = 0.0;
    *vol = 0.0;
    int64_t ci[3] = {0, 0, 0};
    ci[0] = cell % ncell[0];
    ci[1] = (cell / ncell[0]) % ncell[1];
    if (dim == 3) ci[2] = cell / (ncell[0] * ncell[1]);
    /* the cell is [clo, clo + h] per axis: uniform, or between two stretched nodes */
    double clo[3], h[3], zero[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < dim; ++k) {
        if (axis && axis[k]) {
            clo[k] = axis[k][ci[k]];
            h[k] = axis[k][ci[k] + 1] - axis[k][ci[k]];
            TALLY(ORC_OPS_FRAME, 1);
        } else {
            clo[k] = origin[k] + (double)ci[k] * h_uniform[k];
            h[k] = h_uniform[k];
            TALLY(ORC_OPS_FRAME, 2);
        }
    }
    simplex S;
    memset(&S, 0, sizeof(S));
    for (int v = 0; v < na; ++v) {
        const double* p = X + (int64_t)E[e * na + v] * dim;
        for (int k = 0; k < dim; ++k) S.v[v][k] = p[k] - clo[k];
        TALLY(ORC_OPS_FRAME, dim);
    }
    double Minv[4][4];
    if (barycentric_map(dim, S.v, Minv) != ORC_OK) return ORC_EDEGENERATE;
    L0->n = 0;
    int st = slist_push(L0, &S);
    if (st) return st;
    for (int k = 0; k < dim; ++k)
        for (int side = 0; side < 2; ++side) {
            double c = side == 0 ? 0.0 : h[k];
            L1->n = 0;
            for (int64_t i = 0; i < L0->n; ++i) {
                st = split_simplex(dim, &L0->s[i], k, c, side, L1);
                if (st) return st;
            }
            slist tmp = *L0; *L0 = *L1; *L1 = tmp;
        }
    for (int64_t i = 0; i < L0->n; ++i) integrate_simplex(dim, &L0->s[i], Minv, zero, h, block, vol);
    return ORC_OK;
}

/* Blocks of all pairs: blocks[p * (d+1) * 2^d + a * 2^d + b], vols[p].  With
 * ops != NULL the per-thread operation tallies of this call are added into
 * ops[0 .. ORC_OPS_N). */
int orc_pair_blocks_counted(int dim, const int64_t* ncell, const double* origin, const double* h,
                            const double* const* axis, const double* X, const int32_t* E, int64_t n_pairs,
                            const int32_t* pair_elem, const int64_t* pair_cell, double* blocks, double* vols,
                            int nthreads, uint64_t* ops) {
    int nbl = (dim + 1) << dim;
    int status = ORC_OK;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
#endif
    {
        slist L0 = {0, 0, 0}, L1 = {0, 0, 0};
        for (int c = 0; c < ORC_OPS_N; ++c) t_ops[c] = 0;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 256)
#endif
        for (int64_t p = 0; p < n_pairs; ++p) {
            int st = pair_block(dim, ncell, origin, h, axis, X, E, pair_elem[p], pair_cell[p],
                                blocks + p * nbl, vols + p, &L0, &L1);
            if (st) {
#ifdef _OPENMP
#pragma omp critical
#endif
                status = st;
            }
        }
        free(L0.s);
        free(L1.s);
        if (ops) {
#ifdef _OPENMP
#pragma omp critical
#endif
            for (int c = 0; c < ORC_OPS_N; ++c) ops[c] += t_ops[c];
        }
    }
    (void)nthreads;
    return status;
}

int orc_pair_blocks(int dim, const int64_t* ncell, const double* origin, const double* h,
                    const double* const* axis, const double* X, const int32_t* E, int64_t n_pairs,
                    const int32_t* pair_elem, const int64_t* pair_cell, double* blocks, double* vols,
                    int nthreads) {
    return orc_pair_blocks_counted(dim, ncell, origin, h, axis, X, E, n_pairs, pair_elem, pair_cell, blocks, vols,
                                   nthreads, NULL);
}
