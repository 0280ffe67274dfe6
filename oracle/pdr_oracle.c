/*
 * pdr_oracle.c -- plain FP64 CPU oracle for Potential Difference Reduction
 * (PDR) on the multicommodity-flow feasibility problem.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline / reference arm may load or call this library.
 * It shares no source, header, table or constant with the CUDA path.
 *
 * Source: P. Liu, "A Localized Method for Multicommodity Flow Problem"
 * (arXiv 2108.07549).  Every function names the passage it follows.  The
 * code is written for a reader who checks it against the paper by eye: no
 * blocking, no fusion, no reordering beyond what the paper states.
 *
 * Arithmetic: IEEE double, round to nearest, built with -ffp-contract=off so
 * that no multiply-add is fused and results are the same on every host.
 * OpenMP only splits independent per-edge / per-vertex loops; every
 * reduction runs serially in a fixed order, so results do not depend on the
 * thread count.
 *
 * Layout: flows f[e*K + k] (edge-major, commodity-contiguous); heights and
 * excesses h[i*K + k].  Edge e is CSR position e: its tail is the vertex i
 * with row_ptr[i] <= e < row_ptr[i+1], its head is col[e].
 *
 * Readings of passages that are silent or ambiguous:
 *  - vertex degree delta_i = out-degree + in-degree (Table "Notation"; the
 *    convergence proof of Section 4 counts one term per incident edge);
 *  - Alg. 2 takes Case 1 when s <= u (the paper writes s < u; at s = u both
 *    cases give f' = max(0, c), and Case 2's interval test cannot fire);
 *  - when rounding makes Alg. 2's interval test fail for every p, psi is
 *    taken from the active-set rule p* = max{p : c_(p) - cand(p)/2 > 0},
 *    which selects the same p in exact arithmetic; such edges are counted;
 *  - a vertex of degree 0 has h = 0 (it carries no flow and no height);
 *  - a commodity whose origin or destination has degree 0 makes the
 *    instance infeasible outright (no arc can carry its demand).
 */

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Problem description                                                       */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t n;             /* |V| */
    int64_t m;             /* |E| */
    int32_t K;             /* |K| */
    const int64_t *row_ptr;  /* [n+1] out-adjacency (CSR) */
    const int32_t *col;      /* [m] head of edge e */
    const double *u;         /* [m] capacities u_ij */
    const int32_t *s;        /* [K] origins s_k */
    const int32_t *t;        /* [K] destinations t_k */
    const double *d;         /* [K] demands d_k */
    /* filled by orc_adjacency */
    int64_t *in_ptr;   /* [n+1] in-adjacency offsets */
    int64_t *in_eid;   /* [m] edge ids entering each vertex, ascending */
    int32_t *src;      /* [m] tail of edge e */
    int32_t *deg;      /* [n] delta_i = |delta+(i)| + |delta-(i)| */
} orc_problem;

void orc_set_threads(int32_t threads)
{
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
}

int32_t orc_max_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Graph notation (Table "Notation"): delta+(i), delta-(i), delta_i           */
/* ------------------------------------------------------------------------ */

/* Builds the in-adjacency (edges entering each vertex, ascending edge id),
 * the tail of every edge and the degree of every vertex.  Returns 0, or -1 if
 * the CSR is malformed. */
int32_t orc_adjacency(orc_problem *P)
{
    const int32_t n = P->n;
    const int64_t m = P->m;
    if (P->row_ptr[0] != 0 || P->row_ptr[n] != m) return -1;
    for (int32_t i = 0; i < n; ++i) {
        if (P->row_ptr[i + 1] < P->row_ptr[i]) return -1;
        for (int64_t e = P->row_ptr[i]; e < P->row_ptr[i + 1]; ++e) {
            if (P->col[e] < 0 || P->col[e] >= n) return -1;
            P->src[e] = i;
        }
    }
    for (int32_t i = 0; i <= n; ++i) P->in_ptr[i] = 0;
    for (int64_t e = 0; e < m; ++e) P->in_ptr[P->col[e] + 1] += 1;
    for (int32_t i = 0; i < n; ++i) P->in_ptr[i + 1] += P->in_ptr[i];
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!next) return -1;
    for (int32_t i = 0; i < n; ++i) next[i] = P->in_ptr[i];
    for (int64_t e = 0; e < m; ++e) P->in_eid[next[P->col[e]]++] = e;
    free(next);
    for (int32_t i = 0; i < n; ++i) {
        int64_t outdeg = P->row_ptr[i + 1] - P->row_ptr[i];
        int64_t indeg = P->in_ptr[i + 1] - P->in_ptr[i];
        P->deg[i] = (int32_t)(outdeg + indeg);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Excess and height: eq. (3), eq. (3h), eq. (2)                             */
/* ------------------------------------------------------------------------ */

/* Delta_ik = sum_{in-edges} f_{ji,k} - sum_{out-edges} f_{ij,k} + hat-Delta_ik,
 * hat-Delta_ik = d_k at i = s_k, -d_k at i = t_k, 0 elsewhere (eq. (3h)),
 * h_ik = Delta_ik / delta_i.
 * Summation order: in-edges by ascending edge id, then out-edges ascending,
 * then the source/sink term. */
void orc_excess(const orc_problem *P, const double *f, double *Delta, double *h)
{
    const int32_t n = P->n, K = P->K;
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t k = 0; k < K; ++k) {
            double acc = 0.0;
            for (int64_t q = P->in_ptr[i]; q < P->in_ptr[i + 1]; ++q)
                acc += f[P->in_eid[q] * K + k];
            for (int64_t e = P->row_ptr[i]; e < P->row_ptr[i + 1]; ++e)
                acc -= f[e * K + k];
            double hat = 0.0;
            if (i == P->s[k]) hat = P->d[k];
            else if (i == P->t[k]) hat = -P->d[k];
            acc += hat;
            Delta[(int64_t)i * K + k] = acc;
            h[(int64_t)i * K + k] = (P->deg[i] > 0) ? acc / (double)P->deg[i] : 0.0;
        }
    }
}

/* eq. (3), (3h), (2) at one vertex i, reading the flows of edge e from
 * rows[row_of_edge[e]*K ...] (a compact store holding only the rows that
 * are needed; every edge incident to i must be present).  Same summation
 * order as orc_excess.  Returns 0, or -1 if an incident row is missing. */
int32_t orc_excess_vertex(const orc_problem *P, const int64_t *row_of_edge, const double *rows, int32_t i,
                          double *Delta, double *h)
{
    const int32_t K = P->K;
    for (int64_t q = P->in_ptr[i]; q < P->in_ptr[i + 1]; ++q)
        if (row_of_edge[P->in_eid[q]] < 0) return -1;
    for (int64_t e = P->row_ptr[i]; e < P->row_ptr[i + 1]; ++e)
        if (row_of_edge[e] < 0) return -1;
    for (int32_t k = 0; k < K; ++k) {
        double acc = 0.0;
        for (int64_t q = P->in_ptr[i]; q < P->in_ptr[i + 1]; ++q) acc += rows[row_of_edge[P->in_eid[q]] * K + k];
        for (int64_t e = P->row_ptr[i]; e < P->row_ptr[i + 1]; ++e) acc -= rows[row_of_edge[e] * K + k];
        double hat = 0.0;
        if (i == P->s[k]) hat = P->d[k];
        else if (i == P->t[k]) hat = -P->d[k];
        acc += hat;
        Delta[k] = acc;
        h[k] = (P->deg[i] > 0) ? acc / (double)P->deg[i] : 0.0;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Congestion: eq. (41)                                                      */
/* ------------------------------------------------------------------------ */

/* psi_ij = max(0, sum_k f_ij,k - u_ij), summing k in ascending order. */
void orc_congestion(const orc_problem *P, const double *f, double *psi)
{
    const int64_t m = P->m;
    const int32_t K = P->K;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        double tot = 0.0;
        for (int32_t k = 0; k < K; ++k) tot += f[e * K + k];
        double over = tot - P->u[e];
        psi[e] = over > 0.0 ? over : 0.0;
    }
}

/* eq. (41) for one edge from its row of flows. */
double orc_congestion_edge(int32_t K, const double *f_row, double u)
{
    double tot = 0.0;
    for (int32_t k = 0; k < K; ++k) tot += f_row[k];
    double over = tot - u;
    return over > 0.0 ? over : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Objective: Alg. 1 (vertex form) and eq. (8) (edge form)                   */
/* ------------------------------------------------------------------------ */

/* z = 1/2 sum_e psi_e^2 + 1/2 sum_{i,k} delta_i h_ik^2  (Alg. 1). */
double orc_objective(const orc_problem *P, const double *h, const double *psi)
{
    double ze = 0.0, zv = 0.0;
    for (int64_t e = 0; e < P->m; ++e) ze += psi[e] * psi[e];
    for (int32_t i = 0; i < P->n; ++i) {
        double row = 0.0;
        for (int32_t k = 0; k < P->K; ++k) {
            double x = h[(int64_t)i * P->K + k];
            row += x * x;
        }
        zv += (double)P->deg[i] * row;
    }
    return 0.5 * ze + 0.5 * zv;
}

/* z = 1/2 sum_{(i,j)} [psi_ij^2 + sum_k h_ik^2 + sum_k h_jk^2]  (eq. (8)). */
double orc_objective_edges(const orc_problem *P, const double *h, const double *psi)
{
    double z = 0.0;
    for (int64_t e = 0; e < P->m; ++e) {
        const double *hi = h + (int64_t)P->src[e] * P->K;
        const double *hj = h + (int64_t)P->col[e] * P->K;
        double term = psi[e] * psi[e];
        for (int32_t k = 0; k < P->K; ++k) term += hi[k] * hi[k] + hj[k] * hj[k];
        z += term;
    }
    return 0.5 * z;
}

/* ------------------------------------------------------------------------ */
/* Edge subproblem: eq. (10) solved by Alg. 2                                */
/* ------------------------------------------------------------------------ */

static int cmp_desc(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x < y) - (x > y);
}

/* Alg. 2 for one edge (i, j).
 *   hi, hj, f : h_ik, h_jk, f_ij,k for k = 0..K-1
 *   f_new     : f'_ij,k
 *   c, pos    : caller scratch of K doubles each
 * Returns 1 when the active-set rule replaced a failed interval test. */
int32_t orc_edge_qp(int32_t K, const double *hi, const double *hj, const double *f, double u,
                    double *f_new, double *r_out, double *psi_out, double *c, double *pos)
{
    /* 1. preprocessing: c_k = 1/2 ((h_ik + f_k) - (h_jk - f_k)) */
    for (int32_t k = 0; k < K; ++k) c[k] = 0.5 * ((hi[k] + f[k]) - (hj[k] - f[k]));

    /* 2. congestion check: s = sum_k max(0, c_k) */
    double s = 0.0;
    for (int32_t k = 0; k < K; ++k)
        if (c[k] > 0.0) s += c[k];

    double psi = 0.0, r = 0.0;
    int32_t fallback = 0;
    if (s <= u) {
        /* Case 1: uncongested */
        r = u - s;
        psi = 0.0;
    } else {
        /* Case 2: congested; sort the positive potentials in descending order */
        r = 0.0;
        int32_t mp = 0;
        for (int32_t k = 0; k < K; ++k)
            if (c[k] > 0.0) pos[mp++] = c[k];
        qsort(pos, (size_t)mp, sizeof(double), cmp_desc);
        double sum_c = 0.0;
        int32_t found = 0;
        for (int32_t p = 1; p <= mp; ++p) {
            sum_c += pos[p - 1];
            double cand = (sum_c - u) / (1.0 + (double)p / 2.0);
            double upper = pos[p - 1];
            double lower = (p < mp) ? pos[p] : 0.0;
            if (2.0 * lower < cand && cand <= 2.0 * upper) {
                psi = cand;
                found = 1;
                break;
            }
        }
        if (!found) {
            fallback = 1;
            sum_c = 0.0;
            for (int32_t p = 1; p <= mp; ++p) {
                sum_c += pos[p - 1];
                double cand = (sum_c - u) / (1.0 + (double)p / 2.0);
                if (pos[p - 1] - cand / 2.0 > 0.0) psi = cand;
            }
        }
    }

    /* 3. final flows: f'_k = max(0, c_k - psi/2) */
    for (int32_t k = 0; k < K; ++k) {
        double v = c[k] - psi / 2.0;
        f_new[k] = v > 0.0 ? v : 0.0;
    }
    if (r_out) *r_out = r;
    if (psi_out) *psi_out = psi;
    return fallback;
}

/* The QP step of Alg. 1 for every edge, all from the same heights h^(t)
 * (Jacobi: no edge sees another edge's new flow).  f_new may not alias f.
 * Writes the new congestion psi'_e of each subproblem if psi_new != NULL.
 * Returns the number of edges that needed the active-set rule. */
int64_t orc_qp_all(const orc_problem *P, const double *h, const double *f, double *f_new, double *psi_new)
{
    const int64_t m = P->m;
    const int32_t K = P->K;
    int64_t fallbacks = 0;
#pragma omp parallel reduction(+ : fallbacks)
    {
        double *c = (double *)malloc(sizeof(double) * (size_t)K);
        double *pos = (double *)malloc(sizeof(double) * (size_t)K);
#pragma omp for schedule(static)
        for (int64_t e = 0; e < m; ++e) {
            double r, psi;
            fallbacks += orc_edge_qp(K, h + (int64_t)P->src[e] * K, h + (int64_t)P->col[e] * K, f + e * K,
                                     P->u[e], f_new + e * K, &r, &psi, c, pos);
            if (psi_new) psi_new[e] = psi;
        }
        free(c);
        free(pos);
    }
    return fallbacks;
}

/* ------------------------------------------------------------------------ */
/* Capacity kept: Program (6) ("Further Discussion on Optimality Condition") */
/* ------------------------------------------------------------------------ */

/* Program (6) keeps the capacity constraint sum_k f_ij,k <= u_ij and
 * minimises only the height part of the objective, sum_i,k of the integral
 * of h_ik, i.e. 1/2 sum_i,k delta_i h_ik^2 for h = Delta/delta.  The paper
 * gives its KKT conditions (a pipe pressure gamma_ij >= 0 per edge) but no
 * algorithm.  Reading: Alg. 1 with the capacity kept in the local step.
 * Every edge replaces its flows by the minimiser of sum_k (f'_k - c_k)^2
 * over {f' >= 0, sum_k f'_k <= u_ij}, with Alg. 2's c_k = f_k + (h_ik -
 * h_jk)/2; that is eq. (10) with its congestion term replaced by the kept
 * constraint, and it is the Euclidean projection of c onto that set:
 *   f'_k = max(0, c_k - g),  g = 0 if sum_k max(0, c_k) <= u, else the
 *   g > 0 with sum_k max(0, c_k - g) = u.
 * As in Alg. 2, the positive c_k are sorted in descending order and g is
 * the candidate g_p = (sum_{q <= p} c_(q) - u) / p that lies in
 * [c_(p+1), c_(p)] (c_(mp+1) = 0).  A fixed point satisfies the KKT
 * conditions (i)-(iii) of that section with pipe pressure 2g.
 * Returns 1 when rounding made every interval test fail and g was taken as
 * the largest candidate with c_(p) - g_p >= 0. */
int32_t orc_edge_ck(int32_t K, const double *hi, const double *hj, const double *f, double u, double *f_new,
                    double *g_out, double *c, double *pos)
{
    for (int32_t k = 0; k < K; ++k) c[k] = 0.5 * ((hi[k] + f[k]) - (hj[k] - f[k]));
    double s = 0.0;
    for (int32_t k = 0; k < K; ++k)
        if (c[k] > 0.0) s += c[k];
    double g = 0.0;
    int32_t fallback = 0;
    if (s > u) {
        int32_t mp = 0;
        for (int32_t k = 0; k < K; ++k)
            if (c[k] > 0.0) pos[mp++] = c[k];
        qsort(pos, (size_t)mp, sizeof(double), cmp_desc);
        double sum_c = 0.0;
        int32_t found = 0;
        for (int32_t p = 1; p <= mp; ++p) {
            sum_c += pos[p - 1];
            const double cand = (sum_c - u) / (double)p;
            const double lower = (p < mp) ? pos[p] : 0.0;
            if (lower <= cand && cand <= pos[p - 1]) {
                g = cand;
                found = 1;
                break;
            }
        }
        if (!found) {
            fallback = 1;
            sum_c = 0.0;
            for (int32_t p = 1; p <= mp; ++p) {
                sum_c += pos[p - 1];
                const double cand = (sum_c - u) / (double)p;
                if (pos[p - 1] - cand >= 0.0) g = cand;
            }
        }
    }
    for (int32_t k = 0; k < K; ++k) {
        const double v = c[k] - g;
        f_new[k] = v > 0.0 ? v : 0.0;
    }
    if (g_out) *g_out = g;
    return fallback;
}

/* The capacity-kept step for every edge from the same heights h^(t)
 * (Jacobi, as orc_qp_all).  g_new, if not NULL, receives each edge's g.
 * Returns the number of edges that needed the fallback. */
int64_t orc_ck_all(const orc_problem *P, const double *h, const double *f, double *f_new, double *g_new)
{
    const int64_t m = P->m;
    const int32_t K = P->K;
    int64_t fallbacks = 0;
#pragma omp parallel reduction(+ : fallbacks)
    {
        double *c = (double *)malloc(sizeof(double) * (size_t)K);
        double *pos = (double *)malloc(sizeof(double) * (size_t)K);
#pragma omp for schedule(static)
        for (int64_t e = 0; e < m; ++e) {
            double g;
            fallbacks += orc_edge_ck(K, h + (int64_t)P->src[e] * K, h + (int64_t)P->col[e] * K, f + e * K, P->u[e],
                                     f_new + e * K, &g, c, pos);
            if (g_new) g_new[e] = g;
        }
        free(c);
        free(pos);
    }
    return fallbacks;
}

/* ------------------------------------------------------------------------ */
/* Residuals of eq. (1), certificate and verdict                             */
/* ------------------------------------------------------------------------ */

typedef struct {
    double z;            /* Alg. 1 objective at f */
    double cap_abs;      /* max_e max(0, sum_k f_e,k - u_e) */
    double cap_rel;      /* max_e of the same / max(u_e, mean positive u) */
    double cons_abs;     /* max_{i,k} |Delta_ik| */
    double cons_rel;     /* max_{i,k} |Delta_ik| / d_k */
    double f_min;        /* min_{e,k} f_e,k (non-negativity) */
    double margin;       /* Farkas margin, > 0 proves infeasibility */
    double margin_scale; /* magnitude of the margin's terms */
    int32_t verdict;     /* 0 unknown, 1 feasible, 2 infeasible */
    int32_t isolated;    /* 1 if some s_k or t_k has degree 0 */
} orc_residuals;

/* The capacity scale used for edges of zero capacity: the mean positive
 * capacity (1 if no capacity is positive). */
static double capacity_scale(const orc_problem *P)
{
    double tot = 0.0;
    int64_t cnt = 0;
    for (int64_t e = 0; e < P->m; ++e)
        if (P->u[e] > 0.0) {
            tot += P->u[e];
            ++cnt;
        }
    return cnt ? tot / (double)cnt : 1.0;
}

/* Residuals of the three constraint groups of eq. (1) at flows f, plus the
 * Farkas certificate built from the heights (Theorems 1 and 2 say a
 * nonzero-stable pseudo-flow certifies infeasibility).
 *
 * Certificate: potentials pi_ik = h_ik and lengths
 * l_e = max(0, max_k (h_ik - h_jk)) satisfy pi_ik - pi_jk <= l_e, l >= 0.
 * For any feasible flow, sum_k d_k (pi_{s_k,k} - pi_{t_k,k})
 * = sum_{e,k} f_e,k (pi_ik - pi_jk) <= sum_e l_e sum_k f_e,k <= sum_e u_e l_e,
 * so margin = sum_k d_k (h_{s_k,k} - h_{t_k,k}) - sum_e u_e l_e > 0 proves
 * eq. (1) infeasible.
 *
 * Verdict: infeasible if margin > 1e-9 * margin_scale (or an endpoint is
 * isolated); feasible if cap_rel <= tol and cons_rel <= tol; else unknown. */
void orc_residuals_at(const orc_problem *P, const double *f, double tol, orc_residuals *R)
{
    const int32_t n = P->n, K = P->K;
    const int64_t m = P->m;
    double *Delta = (double *)malloc(sizeof(double) * (size_t)n * (size_t)K);
    double *h = (double *)malloc(sizeof(double) * (size_t)n * (size_t)K);
    double *psi = (double *)malloc(sizeof(double) * (size_t)m);
    orc_excess(P, f, Delta, h);
    orc_congestion(P, f, psi);
    R->z = orc_objective(P, h, psi);

    double ubar = capacity_scale(P);
    R->cap_abs = 0.0;
    R->cap_rel = 0.0;
    for (int64_t e = 0; e < m; ++e) {
        double scale = P->u[e] > ubar ? P->u[e] : ubar;
        if (psi[e] > R->cap_abs) R->cap_abs = psi[e];
        if (psi[e] / scale > R->cap_rel) R->cap_rel = psi[e] / scale;
    }
    R->cons_abs = 0.0;
    R->cons_rel = 0.0;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t k = 0; k < K; ++k) {
            double a = fabs(Delta[(int64_t)i * K + k]);
            if (a > R->cons_abs) R->cons_abs = a;
            if (a / P->d[k] > R->cons_rel) R->cons_rel = a / P->d[k];
        }
    R->f_min = m * (int64_t)K > 0 ? f[0] : 0.0;
    for (int64_t q = 0; q < m * (int64_t)K; ++q)
        if (f[q] < R->f_min) R->f_min = f[q];

    double gain = 0.0, gain_abs = 0.0, cost = 0.0;
    for (int32_t k = 0; k < K; ++k) {
        double diff = h[(int64_t)P->s[k] * K + k] - h[(int64_t)P->t[k] * K + k];
        gain += P->d[k] * diff;
        gain_abs += P->d[k] * fabs(diff);
    }
    for (int64_t e = 0; e < m; ++e) {
        const double *hi = h + (int64_t)P->src[e] * K;
        const double *hj = h + (int64_t)P->col[e] * K;
        double l = 0.0;
        for (int32_t k = 0; k < K; ++k)
            if (hi[k] - hj[k] > l) l = hi[k] - hj[k];
        cost += P->u[e] * l;
    }
    R->margin = gain - cost;
    R->margin_scale = gain_abs + cost;

    R->isolated = 0;
    for (int32_t k = 0; k < K; ++k)
        if (P->deg[P->s[k]] == 0 || P->deg[P->t[k]] == 0) R->isolated = 1;

    if (R->isolated || R->margin > 1e-9 * R->margin_scale) R->verdict = 2;
    else if (R->cap_rel <= tol && R->cons_rel <= tol) R->verdict = 1;
    else R->verdict = 0;
    free(Delta);
    free(h);
    free(psi);
}

/* ------------------------------------------------------------------------ */
/* Alg. 1: PDR via exact subproblem optimization                             */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t max_sweeps;   /* max_iterations */
    double eps_obj;       /* stop when |z^(t) - z_prev| < eps_obj; <= 0 disables */
    double resid_tol;     /* also stop when cap_rel, cons_rel <= resid_tol; <= 0 disables */
} orc_options;

typedef struct {
    int64_t sweeps;       /* t at exit: number of QP updates applied */
    double z;             /* z^(t) of the returned flows */
    double z_prev;        /* objective of the sweep before */
    int32_t stop_reason;  /* 0 max_sweeps, 1 objective change, 2 residual target */
    int64_t qp_fallbacks; /* edges where the active-set rule replaced the interval test */
} orc_report;

/* Runs Alg. 1 from the flows in f (the paper starts at f = 0) and leaves
 * f^(t) in f; the local step is Alg. 2 (capacity_kept = 0) or the
 * capacity-kept projection of Program (6) (capacity_kept = 1).  The
 * objective is z = 1/2 sum psi^2 + 1/2 sum delta h^2 in both cases (with the
 * capacity kept, psi = 0 after the first step and z is Program (6)'s).
 * ztrace, if not NULL, receives z^(0..) up to ztrace_len entries.
 * Returns 0, or -1 on allocation failure. */
static int32_t solve_alg1(const orc_problem *P, const orc_options *opt, double *f, orc_report *rep, double *ztrace,
                          int64_t ztrace_len, int capacity_kept)
{
    const int32_t n = P->n, K = P->K;
    const int64_t m = P->m;
    double *Delta = (double *)malloc(sizeof(double) * (size_t)n * (size_t)K);
    double *h = (double *)malloc(sizeof(double) * (size_t)n * (size_t)K);
    double *psi = (double *)malloc(sizeof(double) * (size_t)m);
    double *f_next = (double *)malloc(sizeof(double) * (size_t)m * (size_t)K);
    if (!Delta || !h || !psi || !f_next) {
        free(Delta);
        free(h);
        free(psi);
        free(f_next);
        return -1;
    }
    double ubar = capacity_scale(P);
    double z_prev = INFINITY, z = 0.0;
    int64_t t = 0;
    rep->stop_reason = 0;
    rep->qp_fallbacks = 0;
    for (;;) {
        /* excess and heights, congestion, objective */
        orc_excess(P, f, Delta, h);
        orc_congestion(P, f, psi);
        z = orc_objective(P, h, psi);
        if (ztrace && t < ztrace_len) ztrace[t] = z;
        if (t >= opt->max_sweeps) break;
        /* convergence check on the objective change */
        if (opt->eps_obj > 0.0 && fabs(z - z_prev) < opt->eps_obj) {
            rep->stop_reason = 1;
            break;
        }
        if (opt->resid_tol > 0.0) {
            double cap = 0.0, cons = 0.0;
            for (int64_t e = 0; e < m; ++e) {
                double scale = P->u[e] > ubar ? P->u[e] : ubar;
                if (psi[e] / scale > cap) cap = psi[e] / scale;
            }
            for (int32_t i = 0; i < n; ++i)
                for (int32_t k = 0; k < K; ++k) {
                    double a = fabs(Delta[(int64_t)i * K + k]) / P->d[k];
                    if (a > cons) cons = a;
                }
            if (cap <= opt->resid_tol && cons <= opt->resid_tol) {
                rep->stop_reason = 2;
                break;
            }
        }
        z_prev = z;
        /* update flows by solving every edge subproblem */
        rep->qp_fallbacks += capacity_kept ? orc_ck_all(P, h, f, f_next, NULL) : orc_qp_all(P, h, f, f_next, NULL);
        memcpy(f, f_next, sizeof(double) * (size_t)m * (size_t)K);
        ++t;
    }
    rep->sweeps = t;
    rep->z = z;
    rep->z_prev = z_prev;
    free(Delta);
    free(h);
    free(psi);
    free(f_next);
    return 0;
}

int32_t orc_solve_eso(const orc_problem *P, const orc_options *opt, double *f, orc_report *rep, double *ztrace,
                      int64_t ztrace_len)
{
    return solve_alg1(P, opt, f, rep, ztrace, ztrace_len, 0);
}

/* Alg. 1 with the capacity-kept step (Program (6)); see orc_edge_ck. */
int32_t orc_solve_ck(const orc_problem *P, const orc_options *opt, double *f, orc_report *rep, double *ztrace,
                     int64_t ztrace_len)
{
    return solve_alg1(P, opt, f, rep, ztrace, ztrace_len, 1);
}

/* ------------------------------------------------------------------------ */
/* Alg. 3 (PDR-AGD) and Alg. 4 (PDR-GDM): projected gradient steps          */
/* ------------------------------------------------------------------------ */

/* Parameters of Section 7: AGD beta_init 0.25, beta_min 1/K, beta_max 0.5,
 * alpha_inc 2, alpha_dec 0.5; GDM beta_init 0.1, gamma 0.9, beta_min 1/K,
 * beta_max 0.2, alpha_inc 2, alpha_dec 0.5. */
typedef struct {
    int32_t momentum; /* 0: Alg. 3 (AGD), 1: Alg. 4 (GDM) */
    int32_t pad;
    double beta_init, beta_min, beta_max, alpha_inc, alpha_dec, gamma;
} orc_gd_params;

/* One edge of the update loop of Alg. 3 / Alg. 4 at iteration t.
 *   hi, hj   h_ik, h_jk at iteration t;  psi = psi_ij^(t) (eq. (41))
 *   f, v     flows (and velocities for Alg. 4) of the edge, updated in place
 *   beta     the edge's learning rate, updated in place
 *   df       caller scratch of K doubles
 * Local objective change of the step (eq. (9) with the optimal slack, minus
 * its value at Delta f = 0):
 *   dz = 1/2 (psi'^2 - psi^2) + sum_k (Delta f_k^2 - (h_ik - h_jk) Delta f_k),
 *   psi' = max(0, sum_k (f_k + Delta f_k) - u).
 * Returns 1 if the step was accepted. */
int32_t orc_gd_edge(const orc_gd_params *prm, int32_t K, const double *hi, const double *hj, double psi, double u,
                    double *f, double *v, double *beta, int64_t t, double *df, double *dz_out)
{
    /* potential differences and the projected step */
    double tot = 0.0;
    for (int32_t k = 0; k < K; ++k) {
        double phi = hi[k] - hj[k] - psi;
        double step = *beta * phi;
        df[k] = step > -f[k] ? step : -f[k];
        tot += f[k] + df[k];
    }
    double over = tot - u;
    double psi_new = over > 0.0 ? over : 0.0;
    double dz = 0.5 * (psi_new * psi_new - psi * psi);
    for (int32_t k = 0; k < K; ++k) dz += df[k] * df[k] - (hi[k] - hj[k]) * df[k];
    int32_t accept = dz <= 0.0;
    if (accept) {
        if (prm->momentum) {
            for (int32_t k = 0; k < K; ++k) {
                v[k] = prm->gamma * v[k] + df[k];
                double x = f[k] + v[k];
                f[k] = x > 0.0 ? x : 0.0;
            }
        } else {
            for (int32_t k = 0; k < K; ++k) f[k] = f[k] + df[k];
        }
    } else {
        double b = *beta * prm->alpha_dec;
        *beta = b > prm->beta_min ? b : prm->beta_min;
    }
    if (t % 10 == 0) {
        double b = *beta * prm->alpha_inc;
        *beta = b < prm->beta_max ? b : prm->beta_max;
    }
    if (dz_out) *dz_out = dz;
    return accept;
}

/* Runs Alg. 3 (momentum = 0) or Alg. 4 (momentum = 1) from the flows in f,
 * velocities v and learning rates beta (the paper starts at f = 0, v = 0,
 * beta = beta_init); all three are updated in place and hold the state of
 * iteration t at exit.  Same stop rules and report as orc_solve_eso.
 * Returns 0, or -1 on allocation failure. */
int32_t orc_solve_gd(const orc_problem *P, const orc_options *opt, const orc_gd_params *prm, double *f, double *v,
                     double *beta, orc_report *rep, double *ztrace, int64_t ztrace_len)
{
    const int32_t n = P->n, K = P->K;
    const int64_t m = P->m;
    double *Delta = (double *)malloc(sizeof(double) * (size_t)n * (size_t)K);
    double *h = (double *)malloc(sizeof(double) * (size_t)n * (size_t)K);
    double *psi = (double *)malloc(sizeof(double) * (size_t)m);
    if (!Delta || !h || !psi) {
        free(Delta);
        free(h);
        free(psi);
        return -1;
    }
    double ubar = capacity_scale(P);
    double z_prev = INFINITY, z = 0.0;
    int64_t t = 0;
    rep->stop_reason = 0;
    rep->qp_fallbacks = 0;
    for (;;) {
        orc_excess(P, f, Delta, h);
        orc_congestion(P, f, psi);
        z = orc_objective(P, h, psi);
        if (ztrace && t < ztrace_len) ztrace[t] = z;
        if (t >= opt->max_sweeps) break;
        if (opt->eps_obj > 0.0 && fabs(z - z_prev) < opt->eps_obj) {
            rep->stop_reason = 1;
            break;
        }
        if (opt->resid_tol > 0.0) {
            double cap = 0.0, cons = 0.0;
            for (int64_t e = 0; e < m; ++e) {
                double scale = P->u[e] > ubar ? P->u[e] : ubar;
                if (psi[e] / scale > cap) cap = psi[e] / scale;
            }
            for (int32_t i = 0; i < n; ++i)
                for (int32_t k = 0; k < K; ++k) {
                    double a = fabs(Delta[(int64_t)i * K + k]) / P->d[k];
                    if (a > cons) cons = a;
                }
            if (cap <= opt->resid_tol && cons <= opt->resid_tol) {
                rep->stop_reason = 2;
                break;
            }
        }
        z_prev = z;
        /* every edge steps from the same h^(t), psi^(t) (the edges' rows are
         * disjoint, so updating them in place is the parallel update) */
#pragma omp parallel
        {
            double *df = (double *)malloc(sizeof(double) * (size_t)(K > 0 ? K : 1));
#pragma omp for schedule(static)
            for (int64_t e = 0; e < m; ++e)
                orc_gd_edge(prm, K, h + (int64_t)P->src[e] * K, h + (int64_t)P->col[e] * K, psi[e], P->u[e],
                            f + e * K, v ? v + e * K : NULL, beta + e, t, df, NULL);
            free(df);
        }
        ++t;
    }
    rep->sweeps = t;
    rep->z = z;
    rep->z_prev = z_prev;
    free(Delta);
    free(h);
    free(psi);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Reverse mode through T unrolled sweeps of Alg. 1 (differentiated form)    */
/* ------------------------------------------------------------------------ */

/* L(u, d) = z(f^(T)) with f^(0) = 0 and f^(t+1) = one sweep of Alg. 1 (eq. (3),
 * (2), then Alg. 2 on every edge).  Computes L and its gradient with respect
 * to the capacities u (grad_u[m]) and the demands d (grad_d[K]).
 *
 * Derivatives used (all from the paper's formulas):
 *  - dz/df_e,k = psi_e + h_jk - h_ik (eq. "cpgrad"); dz/du_e = -psi_e;
 *    dz/dd_k = h_{s_k,k} - h_{t_k,k} (d_k enters Delta at s_k with +, at t_k
 *    with -, eq. (3h), and d(1/2 delta h^2)/dDelta = h).
 *  - Alg. 2 output f'_k = max(0, c_k - theta): uncongested (theta = 0):
 *    df'_k/dc_k = [c_k > 0]; congested, A = {c_k > theta},
 *    theta = (sum_A c - u)/(2 + |A|): df'_k/dc_l = [k in A]([k = l] - [l in A]/(2 + |A|)),
 *    df'_k/du = [k in A]/(2 + |A|).
 *  - c_k = f_k + (h_ik - h_jk)/2, h = Delta/delta, Delta linear in f and d.
 * Stores every f^(t) (memory T*m*K doubles: for small instances).
 * Returns 0, or -1 on allocation failure. */
static int32_t adjoint_alg1(const orc_problem *P, int64_t T, double *L_out, double *grad_u, double *grad_d,
                            int capacity_kept)
{
    const int32_t n = P->n, K = P->K;
    const int64_t m = P->m, mk = m * (int64_t)K, nk = (int64_t)n * K;
    double *fs = (double *)calloc((size_t)(T + 1) * (size_t)mk + 1, sizeof(double)); /* f^(0..T) */
    double *Delta = (double *)malloc(sizeof(double) * (size_t)nk + 8);
    double *h = (double *)malloc(sizeof(double) * (size_t)nk + 8);
    double *psi = (double *)malloc(sizeof(double) * (size_t)m + 8);
    double *fbar = (double *)malloc(sizeof(double) * (size_t)mk + 8);   /* dL/df^(t+1), then dL/df^(t) */
    double *cbar = (double *)malloc(sizeof(double) * (size_t)mk + 8);
    double *Dbar = (double *)malloc(sizeof(double) * (size_t)nk + 8);   /* dL/dDelta^(t) */
    double *c = (double *)malloc(sizeof(double) * (size_t)K + 8);
    double *pos = (double *)malloc(sizeof(double) * (size_t)K + 8);
    double *fn = (double *)malloc(sizeof(double) * (size_t)K + 8);
    if (!fs || !Delta || !h || !psi || !fbar || !cbar || !Dbar || !c || !pos || !fn) {
        free(fs); free(Delta); free(h); free(psi); free(fbar); free(cbar); free(Dbar); free(c); free(pos); free(fn);
        return -1;
    }
    /* forward: f^(t+1) from f^(t) */
    for (int64_t t = 0; t < T; ++t) {
        orc_excess(P, fs + t * mk, Delta, h);
        if (capacity_kept) orc_ck_all(P, h, fs + t * mk, fs + (t + 1) * mk, NULL);
        else orc_qp_all(P, h, fs + t * mk, fs + (t + 1) * mk, NULL);
    }
    /* L = z(f^(T)) and its seeds */
    orc_excess(P, fs + T * mk, Delta, h);
    orc_congestion(P, fs + T * mk, psi);
    *L_out = orc_objective(P, h, psi);
    for (int64_t e = 0; e < m; ++e) {
        const double *hi = h + (int64_t)P->src[e] * K, *hj = h + (int64_t)P->col[e] * K;
        for (int32_t k = 0; k < K; ++k) fbar[e * K + k] = psi[e] + hj[k] - hi[k];
        grad_u[e] = -psi[e];
    }
    for (int32_t k = 0; k < K; ++k)
        grad_d[k] = h[(int64_t)P->s[k] * K + k] - h[(int64_t)P->t[k] * K + k];
    /* reverse through the sweeps */
    for (int64_t t = T - 1; t >= 0; --t) {
        const double *f = fs + t * mk;
        orc_excess(P, f, Delta, h);
        /* Alg. 2 backward, edge by edge: fbar holds dL/df^(t+1) */
        for (int64_t e = 0; e < m; ++e) {
            const double *hi = h + (int64_t)P->src[e] * K, *hj = h + (int64_t)P->col[e] * K;
            /* the root theta of the step (Alg. 2: psi'/2; capacity kept: g); both
             * leave c_k = 1/2((h_ik + f_k) - (h_jk - f_k)) in c */
            double theta;
            if (capacity_kept) {
                orc_edge_ck(K, hi, hj, f + e * K, P->u[e], fn, &theta, c, pos);
            } else {
                double r, psi_new;
                orc_edge_qp(K, hi, hj, f + e * K, P->u[e], fn, &r, &psi_new, c, pos);
                theta = psi_new / 2.0;
            }
            int32_t congested = theta > 0.0;
            double Sbar = 0.0;
            int32_t nA = 0;
            for (int32_t k = 0; k < K; ++k) {
                int32_t act = congested ? (c[k] > theta) : (c[k] > 0.0);
                if (act) {
                    Sbar += fbar[e * K + k];
                    ++nA;
                }
            }
            /* Alg. 2: theta = (S_A - u)/(2 + |A|); capacity kept: (S_A - u)/|A|.
             * With the capacity kept and u = 0 the root is max_k c_k and no
             * element is active: f' = 0 near c, so nothing flows back. */
            double corr = (congested && nA > 0) ? Sbar / ((capacity_kept ? 0.0 : 2.0) + (double)nA) : 0.0;
            for (int32_t k = 0; k < K; ++k) {
                int32_t act = congested ? (c[k] > theta) : (c[k] > 0.0);
                cbar[e * K + k] = act ? fbar[e * K + k] - corr : 0.0;
            }
            grad_u[e] += corr;
        }
        /* c = f + (h_i - h_j)/2: hbar_i += cbar/2 on out-edges, hbar_j -= cbar/2 on in-edges;
         * Dbar = hbar / delta */
        for (int32_t i = 0; i < n; ++i)
            for (int32_t k = 0; k < K; ++k) {
                double hb = 0.0;
                for (int64_t e = P->row_ptr[i]; e < P->row_ptr[i + 1]; ++e) hb += 0.5 * cbar[e * K + k];
                for (int64_t q = P->in_ptr[i]; q < P->in_ptr[i + 1]; ++q) hb -= 0.5 * cbar[P->in_eid[q] * K + k];
                Dbar[(int64_t)i * K + k] = P->deg[i] > 0 ? hb / (double)P->deg[i] : 0.0;
            }
        /* Delta = sum_in f - sum_out f + hat-Delta(d) */
        for (int32_t k = 0; k < K; ++k)
            grad_d[k] += Dbar[(int64_t)P->s[k] * K + k] - Dbar[(int64_t)P->t[k] * K + k];
        for (int64_t e = 0; e < m; ++e)
            for (int32_t k = 0; k < K; ++k)
                fbar[e * K + k] = cbar[e * K + k] + Dbar[(int64_t)P->col[e] * K + k] - Dbar[(int64_t)P->src[e] * K + k];
    }
    free(fs); free(Delta); free(h); free(psi); free(fbar); free(cbar); free(Dbar); free(c); free(pos); free(fn);
    return 0;
}

int32_t orc_adjoint_eso(const orc_problem *P, int64_t T, double *L_out, double *grad_u, double *grad_d)
{
    return adjoint_alg1(P, T, L_out, grad_u, grad_d, 0);
}

/* The same through T capacity-kept sweeps (Program (6)): the step's
 * Jacobian on the active set is I - 1 1^T / |A| and df'/du = 1/|A|. */
int32_t orc_adjoint_ck(const orc_problem *P, int64_t T, double *L_out, double *grad_u, double *grad_d)
{
    return adjoint_alg1(P, T, L_out, grad_u, grad_d, 1);
}

/* L(u, d) = z(f^(T)) alone (the forward of the adjoints), for finite differences. */
static double unrolled_objective(const orc_problem *P, int64_t T, int capacity_kept)
{
    const int64_t mk = P->m * (int64_t)P->K, nk = (int64_t)P->n * P->K;
    double *f = (double *)calloc((size_t)mk + 1, sizeof(double));
    double *g = (double *)calloc((size_t)mk + 1, sizeof(double));
    double *Delta = (double *)malloc(sizeof(double) * (size_t)nk + 8);
    double *h = (double *)malloc(sizeof(double) * (size_t)nk + 8);
    double *psi = (double *)malloc(sizeof(double) * (size_t)P->m + 8);
    for (int64_t t = 0; t < T; ++t) {
        orc_excess(P, f, Delta, h);
        if (capacity_kept) orc_ck_all(P, h, f, g, NULL);
        else orc_qp_all(P, h, f, g, NULL);
        double *x = f;
        f = g;
        g = x;
    }
    orc_excess(P, f, Delta, h);
    orc_congestion(P, f, psi);
    double z = orc_objective(P, h, psi);
    free(f); free(g); free(Delta); free(h); free(psi);
    return z;
}

double orc_unrolled_objective(const orc_problem *P, int64_t T) { return unrolled_objective(P, T, 0); }

double orc_unrolled_objective_ck(const orc_problem *P, int64_t T) { return unrolled_objective(P, T, 1); }
