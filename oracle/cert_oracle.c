/*
 * cert_oracle.c -- plain, slow CPU oracle for the certificate-maintenance step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header, table or
 * helper with the CUDA path; it is the definition of what that path computes,
 * written out as directly as possible so that a reader can check it against the
 * paper by eye.
 *
 * Paper: "Repair Entropy in Dynamic Geometric Nearest-Neighbour Structures".
 *   - Certificate (nn_i, d1_i, d2_i), clearance c_i = d2_i - d1_i:  Sec. 2, Def. 1.
 *   - Maximum step eps_t and candidate frontier {i : c_i <= 4 eps_t}:
 *     Sec. 2 (text after Def. 2) and Algorithm 1 (first two statements).
 *   - Index cells, occupied-cell count C, entropy H(F_t):  Sec. 2, Def. 2.
 *   - Exactness of the repaired certificates:  Appendix A, Cor. A.2.
 *
 * Arithmetic (the paper states no precision; these readings are fixed here):
 *   - Squared distance D(i,j) = ((dx*dx + dy*dy) + dz*dz), dx = x_j - x_i, every
 *     operation an IEEE binary32 round-to-nearest operation.  Built with
 *     -ffp-contract=off and without -ffast-math, so no FMA and no reassociation
 *     (x86-64 evaluates float expressions in SSE single precision).
 *   - Top-2 ordering is lexicographic on the key (D, j): equal squared distances
 *     are broken by the lowest index (the paper is silent on ties).
 *   - d_k = sqrtf(D_k), correctly rounded.
 *   - The entropy is evaluated in binary64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* D(i,j) with the fixed operand order: differences are (j - i). */
static float sq_dist(const float *pi, const float *pj, int dim)
{
    float dx = pj[0] - pi[0];
    float dy = pj[1] - pi[1];
    float s = dx * dx + dy * dy;
    if (dim == 3) {
        float dz = pj[2] - pi[2];
        s = s + dz * dz;
    }
    return s;
}

/*
 * Exact top-2 of query i over every j != i (Def. 1, Cor. A.2).
 * Candidates are visited in ascending j, so a strict '<' keeps, among equal D,
 * the one seen first -- the lowest index -- which realises the (D, j)
 * lexicographic order without an explicit index comparison.
 */
static void top2_one(const float *pos, int64_t n, int dim, int64_t i,
                     int32_t *nn, float *d1sq, float *d2sq)
{
    float b1 = INFINITY, b2 = INFINITY;
    int64_t j1 = -1;
    const float *pi = pos + i * dim;
    for (int64_t j = 0; j < n; ++j) {
        if (j == i)
            continue;
        float D = sq_dist(pi, pos + j * dim, dim);
        if (D < b1) {
            b2 = b1;
            b1 = D;
            j1 = j;
        } else if (D < b2) {
            b2 = D;
        }
    }
    *nn = (int32_t)j1;
    *d1sq = b1;
    *d2sq = b2;
}

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* Number of OpenMP threads a parallel region will use (1 without OpenMP). */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Certificates of every point.  pos is [n][dim] float32, n >= 3. Returns 0. */
int oracle_top2(const float *pos, int64_t n, int dim, int32_t *nn, float *d1sq,
                float *d2sq, int nthreads)
{
    if (n < 3 || (dim != 2 && dim != 3))
        return -1;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i)
        top2_one(pos, n, dim, i, nn + i, d1sq + i, d2sq + i);
    return 0;
}

/*
 * The m nearest of point i over every j != i, ascending in the key (D, j):
 * the k-nearest-neighbour certificate one rank further out (the k = 2
 * certificate of Def. 1 is m = 2).  Candidates are visited in ascending j
 * and placed behind every stored key that is <= theirs, so equal D keep
 * the lower index first.  m <= 32.
 */
static void knn_one(const float *pos, int64_t n, int dim, int64_t i, int m, int32_t *idx, float *d2)
{
    float bd[32];
    int32_t bj[32];
    int have = 0;
    const float *pi = pos + i * dim;
    for (int64_t j = 0; j < n; ++j) {
        if (j == i)
            continue;
        float D = sq_dist(pi, pos + j * dim, dim);
        if (have == m && !(D < bd[m - 1]))
            continue;
        int s = have < m ? have++ : m - 1;
        while (s > 0 && D < bd[s - 1]) {
            bd[s] = bd[s - 1];
            bj[s] = bj[s - 1];
            --s;
        }
        bd[s] = D;
        bj[s] = (int32_t)j;
    }
    for (int r = 0; r < m; ++r) {
        idx[i * m + r] = bj[r];
        d2[i * m + r] = bd[r];
    }
}

/* The m nearest of every point, [n][m] row-major.  1 <= m <= 32, n > m.  Returns 0. */
int oracle_knn(const float *pos, int64_t n, int dim, int m, int32_t *idx, float *d2, int nthreads)
{
    if (m < 1 || m > 32 || n <= m || (dim != 2 && dim != 3))
        return -1;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i)
        knn_one(pos, n, dim, i, m, idx, d2);
    return 0;
}

/* Certificates of the listed query points only (a sample of a large scene). */
int oracle_top2_queries(const float *pos, int64_t n, int dim, const int32_t *q,
                        int64_t nq, int32_t *nn, float *d1sq, float *d2sq,
                        int nthreads)
{
    if (n < 3 || (dim != 2 && dim != 3))
        return -1;
    for (int64_t k = 0; k < nq; ++k)
        if (q[k] < 0 || q[k] >= n)
            return -1;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < nq; ++k)
        top2_one(pos, n, dim, q[k], nn + k, d1sq + k, d2sq + k);
    return 0;
}

/* eps_t = max_i ||p'_i - p_i||  (Algorithm 1, first statement). */
float oracle_eps(const float *p_old, const float *p_new, int64_t n, int dim)
{
    float m = 0.0f;
    for (int64_t i = 0; i < n; ++i) {
        float D = sq_dist(p_old + i * dim, p_new + i * dim, dim);
        if (D > m)
            m = D;
    }
    return sqrtf(m);
}

/*
 * Candidate frontier {i : c_i <= 4 eps + tau_i} in ascending index order
 * (Algorithm 1, second statement; Lemma 1 makes every other point safe).
 * tau_i = 2^-20 ((d1_i + d2_i) + eps) is the rounding guard: Lemma 1 holds in
 * real arithmetic, while the certificates are built from rounded distances.
 * With guard == 0 the bare rule c_i <= 4 eps is applied.
 * Returns the number of frontier points written to out.
 */
int64_t oracle_frontier(const float *d1sq, const float *d2sq, int64_t n, float eps,
                        int guard, int32_t *out)
{
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        float d1 = sqrtf(d1sq[i]);
        float d2 = sqrtf(d2sq[i]);
        float c = d2 - d1;
        float tau = guard ? 0x1p-20f * ((d1 + d2) + eps) : 0.0f;
        float rhs = 4.0f * eps + tau;
        if (c <= rhs)
            out[k++] = (int32_t)i;
    }
    return k;
}

/*
 * Per-point displacement delta_i = sqrtf(|p'_i - p_i|^2), the squared distance
 * in the fixed order above (new minus old).
 */
void oracle_disp(const float *p_old, const float *p_new, int64_t n, int dim, float *out)
{
    for (int64_t i = 0; i < n; ++i)
        out[i] = sqrtf(sq_dist(p_old + i * dim, p_new + i * dim, dim));
}

/*
 * Frontier under the per-point motion budget (the remark closing Sec. 5 on
 * the validity radius): nn_i can change only if some other point gets closer
 * than nn_i; each distance from i changes by at most delta_i + delta_j <=
 * delta_i + eps (triangle inequality, as in Lemma 1), so the certificate is
 * safe when c_i > 2 (delta_i + eps).  Same rounding guard as oracle_frontier.
 */
/*
 * The local heuristic of Sec. 3 and Table 1: point i is flagged when
 * rho_i = delta_i / c_i > 1/2, delta_i its own displacement and c_i = d2_i - d1_i
 * its pre-step clearance.  Written as 2 delta_i > c_i, the same comparison of
 * the FP32 values without rounding a quotient (2 delta_i is exact); c_i = 0
 * with delta_i = 0 (0/0) is not flagged.  Unlike the rules above it is no
 * bound: a point that stays put can still lose its nearest neighbour.
 */
int64_t oracle_rho(const float *d1sq, const float *d2sq, const float *disp, int64_t n, uint8_t *out)
{
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        float c = sqrtf(d2sq[i]) - sqrtf(d1sq[i]);
        out[i] = (uint8_t)(2.0f * disp[i] > c);
        k += out[i];
    }
    return k;
}

int64_t oracle_frontier_point(const float *d1sq, const float *d2sq, const float *disp, int64_t n, float eps,
                              int32_t *out)
{
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        float d1 = sqrtf(d1sq[i]);
        float d2 = sqrtf(d2sq[i]);
        float c = d2 - d1;
        float tau = 0x1p-20f * ((d1 + d2) + eps);
        float rhs = 2.0f * (disp[i] + eps) + tau;
        if (c <= rhs)
            out[k++] = (int32_t)i;
    }
    return k;
}

/* Cells per axis of the entropy grid: the smallest g with g^dim >= n, so the
 * mean occupancy is at most a small constant (Sec. 2, first paragraph). */
int oracle_grid_res(int64_t n, int dim)
{
    int g = 1;
    for (;;) {
        int64_t p = 1;
        for (int a = 0; a < dim; ++a)
            p *= g;
        if (p >= n)
            return g;
        ++g;
    }
}

/* Index cell of every point: per axis k = floor(x * g) clamped to [0, g-1],
 * cell = (kz * g + ky) * g + kx  (kz absent in 2-D). */
void oracle_cells(const float *pos, int64_t n, int dim, int g, int32_t *cell)
{
    float gf = (float)g;
    for (int64_t i = 0; i < n; ++i) {
        int32_t k[3] = {0, 0, 0};
        for (int a = 0; a < dim; ++a) {
            float t = pos[i * dim + a] * gf;
            int32_t v;
            if (!(t >= 0.0f))
                v = 0;
            else if (t >= gf)
                v = g - 1;
            else
                v = (int32_t)floorf(t);
            k[a] = v;
        }
        cell[i] = (dim == 3) ? (k[2] * g + k[1]) * g + k[0] : k[1] * g + k[0];
    }
}

/*
 * Normalised entropy of a point subset over the index cells (Def. 2):
 *   H = -sum_k q_k ln q_k / ln C,   q_k = (members in cell k) / (members),
 * C = number of cells holding at least one of the n points (the occupied cells).
 * The ratio is base-free, so the natural log is used.  When the subset has at
 * most one member, or C <= 1, the value is 0 (a single cell is "localized").
 * Outputs: *m_out = cells the subset meets, *c_out = C.  binary64 throughout.
 */
double oracle_entropy(const int32_t *cell, const uint8_t *member, int64_t n,
                      int64_t ncells, int64_t *m_out, int64_t *c_out)
{
    int64_t *all = calloc((size_t)ncells, sizeof(int64_t));
    int64_t *sub = calloc((size_t)ncells, sizeof(int64_t));
    if (!all || !sub) {
        free(all);
        free(sub);
        return NAN;
    }
    int64_t nsub = 0;
    for (int64_t i = 0; i < n; ++i) {
        all[cell[i]] += 1;
        if (member[i]) {
            sub[cell[i]] += 1;
            nsub += 1;
        }
    }
    int64_t C = 0, m = 0;
    for (int64_t k = 0; k < ncells; ++k) {
        if (all[k] > 0)
            C += 1;
        if (sub[k] > 0)
            m += 1;
    }
    double H = 0.0;
    if (nsub > 1 && C > 1) {
        double s = 0.0;
        for (int64_t k = 0; k < ncells; ++k) {
            if (sub[k] > 0) {
                double q = (double)sub[k] / (double)nsub;
                s -= q * log(q);
            }
        }
        H = s / log((double)C);
    }
    free(all);
    free(sub);
    if (m_out)
        *m_out = m;
    if (c_out)
        *c_out = C;
    return H;
}
