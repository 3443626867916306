/*
 * CPU oracle for the dipolar Barnes-Hut ferrofluid step.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header or
 * constant table with the CUDA library.
 *
 * Everything here follows the paper (Polyakov et al., "Large-scale Ferrofluid
 * Simulations on Graphics Processing Units"), Sections 2-3 and 5:
 *   - reduced dipolar field and force of a pair: Sec. 2, Eqs. (h_dip_red) and
 *     (f_dip) in reduced units;
 *   - Lennard-Jones short-range force: Sec. 2, Eq. (LJ) / reduced f_sr;
 *   - all-pairs sum: Sec. 3.1, Algorithm 1 (plain double loop, self skipped);
 *   - Barnes-Hut octree, pseudo-particle (Eq. magCenter) and traversal:
 *     Sec. 3.2;
 *   - Euler-Maruyama step with dt = 1e-3: Sec. 4;
 *   - magnetisation observables: Sec. 5.
 *
 * Readings where the paper is silent or garbled (opening rule, rotational
 * dynamics in vector form, noise strength 2 kT Gamma_r, wall potential,
 * Philox counter layout, Morton quantisation, aggregation order) are listed
 * with the CUDA design notes; they are restated at each function below.
 *
 * Floating point: all sums are FP64.  The Barnes-Hut *tree* (Morton
 * quantisation, cell centres used for the opening test, the opening decision
 * itself) is computed in the tree precision `prec` (0 = IEEE single, 1 = IEEE
 * double, 2 = mixed: single, except that each cell centre is the FP64
 * position sum divided by the count, rounded once to single) because these
 * floating-point values decide discrete outcomes (which cell a particle falls
 * in, whether a cell is accepted); the paper ran in single precision.  Build with -ffp-contract=off and without fast-math so
 * every single operation is rounded exactly once in the written order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define ORA_MAXLEVEL 21               /* 21 bits per axis -> 63-bit keys */
#define ORA_QMAX ((1u << 21) - 1u)

/* ------------------------------------------------------------------------ */
/* threads                                                                   */
/* ------------------------------------------------------------------------ */
void ora_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int ora_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* pair terms                                                                */
/* ------------------------------------------------------------------------ */
static double dot3(const double *a, const double *b)
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/*
 * Reduced dipolar field of particle j at particle k and the reduced dipolar
 * force on k (Sec. 2, reduced Eqs. h_dip and f_dip):
 *   h = [3 r (u_j.r) - u_j r^2] / r^5
 *   f = 3 [r (u_j.u_k) + u_k (u_j.r) + u_j (u_k.r)] / r^5
 *       - 15 r (u_k.r)(u_j.r) / r^7
 * with r = rho_k - rho_j.  The force expression is written so that swapping
 * (k, j) negates it bit for bit (every product and the inner sum commute).
 * Coincident particles (r = 0) have no defined pair term; the caller skips
 * them.
 */
void ora_pair_dipole(const double r[3], const double uk[3], const double uj[3],
                     double h[3], double f[3])
{
    double r2 = dot3(r, r);
    double ir = 1.0 / sqrt(r2);
    double ir2 = ir * ir;
    double ir3 = ir2 * ir;
    double ir5 = ir3 * ir2;
    double ir7 = ir5 * ir2;
    double bj = dot3(uj, r);
    double bk = dot3(uk, r);
    double a = dot3(uj, uk);
    for (int c = 0; c < 3; ++c) {
        h[c] = (3.0 * r[c] * bj - uj[c] * r2) * ir5;
        f[c] = 3.0 * (r[c] * a + (uk[c] * bj + uj[c] * bk)) * ir5
             - 15.0 * r[c] * (bk * bj) * ir7;
    }
}

/*
 * Reduced Lennard-Jones force as printed (Sec. 2, Eq. LJ / reduced f_sr):
 *   f = 24 eps r / r^2 [(sigma/r)^12 - (sigma/r)^6],   |r| < rcut, else 0.
 * Its pair energy is 2 eps (sigma/r)^12 - 4 eps (sigma/r)^6, shifted to zero
 * at rcut (the printed force is minus the derivative of that energy).
 * Returns the shifted pair energy.
 */
double ora_pair_lj(const double r[3], double eps, double sigma, double rcut,
                   double f[3])
{
    double r2 = dot3(r, r);
    f[0] = f[1] = f[2] = 0.0;
    if (!(r2 < rcut * rcut) || r2 == 0.0) return 0.0;
    double s2 = sigma * sigma / r2;
    double s6 = s2 * s2 * s2;
    double s12 = s6 * s6;
    double coef = 24.0 * eps * (s12 - s6) / r2;
    for (int c = 0; c < 3; ++c) f[c] = coef * r[c];
    double sc2 = sigma * sigma / (rcut * rcut);
    double sc6 = sc2 * sc2 * sc2;
    double shift = 2.0 * eps * sc6 * sc6 - 4.0 * eps * sc6;
    return 2.0 * eps * s12 - 4.0 * eps * s6 - shift;
}

/*
 * Whether a pair lies inside the LJ cut-off, decided in the given precision
 * (0 single, 1 double) with each operation rounded once:
 * r2 = (dx*dx + dy*dy) + dz*dz < rcut^2, with the differences formed in that
 * precision.  The cut decides a discrete outcome, so it is taken in the
 * precision of the arithmetic under test.
 */
static int lj_inside(const double xk[3], const double xj[3], double rcut, int prec)
{
    if (prec != 1) {
        float d[3];
        for (int a = 0; a < 3; ++a) d[a] = (float)xk[a] - (float)xj[a];
        float dxx = d[0] * d[0], dyy = d[1] * d[1], dzz = d[2] * d[2];
        float r2 = dxx + dyy;
        r2 = r2 + dzz;
        float rc2 = (float)(rcut * rcut);
        return r2 < rc2 && r2 > 0.0f;
    }
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = xk[a] - xj[a];
    double r2 = d[0] * d[0] + d[1] * d[1];
    r2 = r2 + d[2] * d[2];
    return r2 < rcut * rcut && r2 > 0.0;
}

/* LJ force and shifted pair energy for a pair already known to be inside the cut */
static double lj_pair_inside(const double r[3], double eps, double sigma, double rcut, double f[3])
{
    double r2 = dot3(r, r);
    double s2 = sigma * sigma / r2;
    double s6 = s2 * s2 * s2;
    double s12 = s6 * s6;
    double coef = 24.0 * eps * (s12 - s6) / r2;
    for (int c = 0; c < 3; ++c) f[c] = coef * r[c];
    double sc2 = sigma * sigma / (rcut * rcut);
    double sc6 = sc2 * sc2 * sc2;
    double shift = 2.0 * eps * sc6 * sc6 - 4.0 * eps * sc6;
    return 2.0 * eps * s12 - 4.0 * eps * s6 - shift;
}

/* ------------------------------------------------------------------------ */
/* all pairs (Sec. 3.1, Algorithm 1)                                         */
/* ------------------------------------------------------------------------ */
/*
 * For every particle k: h_k = dip_scale * sum_{j != k} h_kj,
 * f_k = dip_scale * sum_{j != k} f_kj (+ sum_{j != k} f^sr_kj if
 * include_sr and eps != 0).  e_sr[k] (if non-NULL) receives half of the
 * shifted LJ energy of every pair k is in.  pos, u, h, f are n x 3 row-major.
 * cut_prec: precision in which the LJ cut-off test is taken (0 single,
 * 1 double).  With `only` (n_only indices), only those targets are summed
 * (every other particle is still a source); other rows are left untouched.
 */
void ora_allpairs(int64_t n, const double *pos, const double *u,
                  double dip_scale, double eps, double sigma, double rcut,
                  int32_t include_sr, int32_t cut_prec, const int64_t *only, int64_t n_only,
                  double *h, double *f, double *e_sr)
{
    int use_lj = include_sr && eps != 0.0 && rcut > 0.0;
    int64_t cnt = only ? n_only : n;
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t q = 0; q < cnt; ++q) {
        int64_t k = only ? only[q] : q;
        double hk[3] = {0, 0, 0}, fd[3] = {0, 0, 0}, fs[3] = {0, 0, 0};
        double ek = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == k) continue;
            double r[3] = {pos[3 * k] - pos[3 * j], pos[3 * k + 1] - pos[3 * j + 1],
                           pos[3 * k + 2] - pos[3 * j + 2]};
            if (dot3(r, r) == 0.0) continue;
            double hp[3], fp[3];
            ora_pair_dipole(r, &u[3 * k], &u[3 * j], hp, fp);
            for (int c = 0; c < 3; ++c) { hk[c] += hp[c]; fd[c] += fp[c]; }
            if (use_lj && lj_inside(&pos[3 * k], &pos[3 * j], rcut, cut_prec)) {
                double fl[3];
                ek += 0.5 * lj_pair_inside(r, eps, sigma, rcut, fl);
                for (int c = 0; c < 3; ++c) fs[c] += fl[c];
            }
        }
        for (int c = 0; c < 3; ++c) {
            h[3 * k + c] = dip_scale * hk[c];
            f[3 * k + c] = dip_scale * fd[c] + fs[c];
        }
        if (e_sr) e_sr[k] = ek;
    }
}

/* ------------------------------------------------------------------------ */
/* Morton keys                                                               */
/* ------------------------------------------------------------------------ */
/*
 * Root cube (kernel 1 of Sec. 3.2): origin = per-axis minimum, side = the
 * largest extent (1 if every extent is zero).  Quantisation, in the tree
 * precision and with each operation rounded once:
 *   q_a = min(floor((x_a - min_a) * S), 2^21 - 1),   S = 2^21 / side.
 * The 63-bit key interleaves the 21 bits of (q_x, q_y, q_z), most significant
 * first, x highest within each 3-bit digit, so the digit at level L (root =
 * level 0) is bits 3(21-L)+2 .. 3(21-L) and names the octant x*4 + y*2 + z.
 */
static uint64_t interleave3(uint32_t qx, uint32_t qy, uint32_t qz)
{
    uint64_t key = 0;
    for (int b = 0; b < 21; ++b) {
        key |= (uint64_t)((qx >> b) & 1u) << (3 * b + 2);
        key |= (uint64_t)((qy >> b) & 1u) << (3 * b + 1);
        key |= (uint64_t)((qz >> b) & 1u) << (3 * b);
    }
    return key;
}

static uint32_t quant_f(float x, float mn, float S)
{
    float t = x - mn;
    float s = t * S;
    float fl = floorf(s);
    if (!(fl > 0.0f)) return 0u;
    if (fl >= 2097151.0f) return ORA_QMAX;
    return (uint32_t)fl;
}

static uint32_t quant_d(double x, double mn, double S)
{
    double t = x - mn;
    double s = t * S;
    double fl = floor(s);
    if (!(fl > 0.0)) return 0u;
    if (fl >= 2097151.0) return ORA_QMAX;
    return (uint32_t)fl;
}

/* root[0..2] = origin, root[3] = side (values of the tree precision) */
void ora_morton(int64_t n, const double *pos, int32_t prec, uint64_t *keys, double root[4])
{
    if (prec != 1) {
        float mn[3], mx[3];
        for (int a = 0; a < 3; ++a) { mn[a] = (float)pos[a]; mx[a] = (float)pos[a]; }
        for (int64_t i = 1; i < n; ++i)
            for (int a = 0; a < 3; ++a) {
                float x = (float)pos[3 * i + a];
                if (x < mn[a]) mn[a] = x;
                if (x > mx[a]) mx[a] = x;
            }
        float side = mx[0] - mn[0];
        for (int a = 1; a < 3; ++a) { float e = mx[a] - mn[a]; if (e > side) side = e; }
        if (!(side > 0.0f)) side = 1.0f;
        float S = 2097152.0f / side;
        for (int64_t i = 0; i < n; ++i) {
            uint32_t q[3];
            for (int a = 0; a < 3; ++a) q[a] = quant_f((float)pos[3 * i + a], mn[a], S);
            keys[i] = interleave3(q[0], q[1], q[2]);
        }
        for (int a = 0; a < 3; ++a) root[a] = mn[a];
        root[3] = side;
    } else {
        double mn[3], mx[3];
        for (int a = 0; a < 3; ++a) { mn[a] = pos[a]; mx[a] = pos[a]; }
        for (int64_t i = 1; i < n; ++i)
            for (int a = 0; a < 3; ++a) {
                double x = pos[3 * i + a];
                if (x < mn[a]) mn[a] = x;
                if (x > mx[a]) mx[a] = x;
            }
        double side = mx[0] - mn[0];
        for (int a = 1; a < 3; ++a) { double e = mx[a] - mn[a]; if (e > side) side = e; }
        if (!(side > 0.0)) side = 1.0;
        double S = 2097152.0 / side;
        for (int64_t i = 0; i < n; ++i) {
            uint32_t q[3];
            for (int a = 0; a < 3; ++a) q[a] = quant_d(pos[3 * i + a], mn[a], S);
            keys[i] = interleave3(q[0], q[1], q[2]);
        }
        for (int a = 0; a < 3; ++a) root[a] = mn[a];
        root[3] = side;
    }
}

/* sort by (key, input index): kernel 4 of Sec. 3.2, stable */
typedef struct { uint64_t key; int64_t idx; } ora_kv;

static int cmp_kv(const void *a, const void *b)
{
    const ora_kv *x = (const ora_kv *)a, *y = (const ora_kv *)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/* ------------------------------------------------------------------------ */
/* octree (Sec. 3.2)                                                         */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n, cap;
    int32_t *level, *leaf;
    int64_t *pbegin, *pend, *skip;
    /* geometry in the tree precision, stored as double */
    double *lo;          /* 3 per cell: lower corner of the dyadic cube */
    double *side;        /* cube side */
    /* aggregates */
    double *S64, *U64;   /* 3 per cell: sum of positions, sum of moments */
    float *S32;          /* 3 per cell: single-precision position sums   */
    double *cen;         /* 3 per cell: pseudo-particle centre used by the tree precision */
} ora_tree_t;

static void tree_push(ora_tree_t *t)
{
    if (t->n < t->cap) return;
    int64_t nc = t->cap ? 2 * t->cap : 1024;
    t->level = realloc(t->level, nc * sizeof(int32_t));
    t->leaf = realloc(t->leaf, nc * sizeof(int32_t));
    t->pbegin = realloc(t->pbegin, nc * sizeof(int64_t));
    t->pend = realloc(t->pend, nc * sizeof(int64_t));
    t->skip = realloc(t->skip, nc * sizeof(int64_t));
    t->cap = nc;
}

static void tree_free(ora_tree_t *t)
{
    free(t->level); free(t->leaf); free(t->pbegin); free(t->pend); free(t->skip);
    free(t->lo); free(t->side); free(t->S64); free(t->U64); free(t->S32); free(t->cen);
    memset(t, 0, sizeof(*t));
}

/*
 * Recursive top-down decomposition (Sec. 3.2): a cell covering sorted
 * particles [b, e) at level L is a leaf if it holds at most leaf_max
 * particles (the paper: one) or L = 21 (keys exhausted; coincident particles
 * stay together); otherwise it is split into its non-empty octants, visited
 * in octant order 0..7, which are maximal runs of equal level-(L+1) digits.
 * Cells are recorded in depth-first preorder; skip = index of the first cell
 * after the subtree.
 */
static void build_rec(const uint64_t *skeys, int64_t b, int64_t e, int L, int leaf_max,
                      ora_tree_t *t)
{
    tree_push(t);
    int64_t idx = t->n++;
    t->level[idx] = L;
    t->pbegin[idx] = b;
    t->pend[idx] = e;
    if (e - b <= leaf_max || L == ORA_MAXLEVEL) {
        t->leaf[idx] = 1;
    } else {
        t->leaf[idx] = 0;
        int shift = 3 * (ORA_MAXLEVEL - (L + 1));
        int64_t s = b;
        while (s < e) {
            uint64_t d = (skeys[s] >> shift) & 7u;
            int64_t s2 = s;
            while (s2 < e && ((skeys[s2] >> shift) & 7u) == d) ++s2;
            build_rec(skeys, s, s2, L + 1, leaf_max, t);
            s = s2;
        }
    }
    t->skip[idx] = t->n;
}

/* de-interleave the level-L prefix of a key into cube coordinates */
static void prefix_coords(uint64_t key, int L, uint32_t q[3])
{
    q[0] = q[1] = q[2] = 0;
    for (int l = 1; l <= L; ++l) {
        int shift = 3 * (ORA_MAXLEVEL - l);
        uint32_t d = (uint32_t)((key >> shift) & 7u);
        q[0] = (q[0] << 1) | ((d >> 2) & 1u);
        q[1] = (q[1] << 1) | ((d >> 1) & 1u);
        q[2] = (q[2] << 1) | (d & 1u);
    }
}

/*
 * Builds keys, order (sorted position -> input index) and the tree.
 * Geometry of a level-L cell with integer cube coordinates q:
 *   side_L = side * 2^-L,  lo_a = origin_a + q_a * side_L
 * (each operation rounded once in the tree precision).
 * Aggregates (Eq. magCenter): n = particle count, U = sum of moments,
 * centre = (sum of positions) / n.  Sums run over a leaf's particles in
 * sorted order and over an internal cell's children in octant order, each
 * partial sum starting from the first term.  The FP64 sums give the exact
 * reference; in single precision the same order is used so the centre that
 * enters the opening test is a defined single-precision number.
 */
static void tree_build(int64_t n, const double *pos, const double *u, int prec,
                       int leaf_max, uint64_t *skeys, int64_t *order, double root[4],
                       ora_tree_t *t)
{
    uint64_t *keys = malloc(n * sizeof(uint64_t));
    ora_morton(n, pos, prec, keys, root);
    ora_kv *kv = malloc(n * sizeof(ora_kv));
    for (int64_t i = 0; i < n; ++i) { kv[i].key = keys[i]; kv[i].idx = i; }
    qsort(kv, (size_t)n, sizeof(ora_kv), cmp_kv);
    for (int64_t i = 0; i < n; ++i) { skeys[i] = kv[i].key; order[i] = kv[i].idx; }
    free(kv);
    free(keys);

    memset(t, 0, sizeof(*t));
    build_rec(skeys, 0, n, 0, leaf_max, t);
    int64_t nc = t->n;
    t->lo = malloc(3 * nc * sizeof(double));
    t->side = malloc(nc * sizeof(double));
    t->S64 = malloc(3 * nc * sizeof(double));
    t->U64 = malloc(3 * nc * sizeof(double));
    t->S32 = malloc(3 * nc * sizeof(float));
    t->cen = malloc(3 * nc * sizeof(double));

    for (int64_t c = 0; c < nc; ++c) {
        uint32_t q[3];
        int L = t->level[c];
        prefix_coords(skeys[t->pbegin[c]], L, q);
        if (prec != 1) {
            float side = ldexpf((float)root[3], -L);
            t->side[c] = side;
            for (int a = 0; a < 3; ++a) {
                float off = (float)q[a] * side;
                float lo = (float)root[a] + off;
                t->lo[3 * c + a] = lo;
            }
        } else {
            double side = ldexp(root[3], -L);
            t->side[c] = side;
            for (int a = 0; a < 3; ++a) {
                double off = (double)q[a] * side;
                t->lo[3 * c + a] = root[a] + off;
            }
        }
    }

    /* bottom-up: in preorder every child has a larger index than its parent */
    for (int64_t c = nc - 1; c >= 0; --c) {
        double S[3], U[3];
        float S32[3];
        if (t->leaf[c]) {
            int64_t j0 = order[t->pbegin[c]];
            for (int a = 0; a < 3; ++a) {
                S[a] = pos[3 * j0 + a];
                U[a] = u[3 * j0 + a];
                S32[a] = (float)pos[3 * j0 + a];
            }
            for (int64_t s = t->pbegin[c] + 1; s < t->pend[c]; ++s) {
                int64_t j = order[s];
                for (int a = 0; a < 3; ++a) {
                    S[a] += pos[3 * j + a];
                    U[a] += u[3 * j + a];
                    S32[a] = S32[a] + (float)pos[3 * j + a];
                }
            }
        } else {
            int64_t ch = c + 1;
            for (int a = 0; a < 3; ++a) {
                S[a] = t->S64[3 * ch + a];
                U[a] = t->U64[3 * ch + a];
                S32[a] = t->S32[3 * ch + a];
            }
            ch = t->skip[ch];
            while (ch < t->skip[c]) {
                for (int a = 0; a < 3; ++a) {
                    S[a] += t->S64[3 * ch + a];
                    U[a] += t->U64[3 * ch + a];
                    S32[a] = S32[a] + t->S32[3 * ch + a];
                }
                ch = t->skip[ch];
            }
        }
        int64_t cnt = t->pend[c] - t->pbegin[c];
        for (int a = 0; a < 3; ++a) {
            t->S64[3 * c + a] = S[a];
            t->U64[3 * c + a] = U[a];
            t->S32[3 * c + a] = S32[a];
            if (prec == 0)
                t->cen[3 * c + a] = (double)(S32[a] / (float)cnt);
            else if (prec == 2)
                t->cen[3 * c + a] = (double)(float)(S[a] / (double)cnt);
            else
                t->cen[3 * c + a] = S[a] / (double)cnt;
        }
    }
}

/*
 * Tree introspection for the topology and aggregation tests.  Returns the
 * number of cells; if it exceeds cap nothing but keys/order/root is written.
 * cen: the centre in the tree precision; c64: the FP64 centre S64/n.
 */
int64_t ora_tree(int64_t n, const double *pos, const double *u, int32_t prec, int32_t leaf_max,
                 uint64_t *skeys, int64_t *order, double root[4], int64_t cap,
                 int32_t *level, int32_t *leaf, int64_t *pbegin, int64_t *pend, int64_t *skip,
                 double *lo, double *side, double *cen, double *c64, double *U64)
{
    ora_tree_t t;
    tree_build(n, pos, u, prec, leaf_max, skeys, order, root, &t);
    int64_t nc = t.n;
    if (nc <= cap) {
        for (int64_t c = 0; c < nc; ++c) {
            level[c] = t.level[c];
            leaf[c] = t.leaf[c];
            pbegin[c] = t.pbegin[c];
            pend[c] = t.pend[c];
            skip[c] = t.skip[c];
            side[c] = t.side[c];
            double cnt = (double)(t.pend[c] - t.pbegin[c]);
            for (int a = 0; a < 3; ++a) {
                lo[3 * c + a] = t.lo[3 * c + a];
                cen[3 * c + a] = t.cen[3 * c + a];
                c64[3 * c + a] = t.S64[3 * c + a] / cnt;
                U64[3 * c + a] = t.U64[3 * c + a];
            }
        }
    }
    tree_free(&t);
    return nc;
}

/* ------------------------------------------------------------------------ */
/* Barnes-Hut traversal (Sec. 3.2)                                           */
/* ------------------------------------------------------------------------ */
typedef struct {
    double theta;
    int32_t leaf_max;
    int32_t prec;          /* tree precision: 0 single, 1 double, 2 mixed */
    double dip_scale;
    double lj_eps, lj_sigma, lj_rcut;
    int32_t include_sr;
    int32_t quad;          /* 1: add each accepted cell's dipole-position (quadrupole) term */
} ora_bh_params;

/*
 * Opening test (the paper only says "far enough"; reading): a cell C is used
 * as its pseudo-particle for particle k iff
 *   (1) k is not one of C's particles,
 *   (2) side_C^2 < theta^2 * |rho_k - centre_C|^2   (strict), and
 *   (3) when the LJ term is on, the distance from rho_k to C's cube is at
 *       least rcut, so every pair closer than rcut is summed exactly.
 * Evaluated in the tree precision, each operation rounded once, in this
 * order: d^2 = (dx*dx + dy*dy) + dz*dz; box distance per axis
 * max(max(lo - x, 0), x - (lo + side)).
 */
static int accept_f(const float xk[3], const float c[3], float side, const float lo[3],
                    float theta2, int use_rcut, float rcut2)
{
    float dx = xk[0] - c[0], dy = xk[1] - c[1], dz = xk[2] - c[2];
    float dxx = dx * dx, dyy = dy * dy, dzz = dz * dz;
    float d2 = dxx + dyy;
    d2 = d2 + dzz;
    float s2 = side * side;
    float td = theta2 * d2;
    if (!(s2 < td)) return 0;
    if (use_rcut) {
        float t[3];
        for (int a = 0; a < 3; ++a) {
            float hi = lo[a] + side;
            float below = lo[a] - xk[a];
            float above = xk[a] - hi;
            float m = below > 0.0f ? below : 0.0f;
            t[a] = above > m ? above : m;
        }
        float txx = t[0] * t[0], tyy = t[1] * t[1], tzz = t[2] * t[2];
        float b2 = txx + tyy;
        b2 = b2 + tzz;
        if (b2 < rcut2) return 0;
    }
    return 1;
}

static int accept_d(const double xk[3], const double c[3], double side, const double lo[3],
                    double theta2, int use_rcut, double rcut2)
{
    double dx = xk[0] - c[0], dy = xk[1] - c[1], dz = xk[2] - c[2];
    double d2 = dx * dx + dy * dy;
    d2 = d2 + dz * dz;
    double s2 = side * side;
    if (!(s2 < theta2 * d2)) return 0;
    if (use_rcut) {
        double t[3];
        for (int a = 0; a < 3; ++a) {
            double hi = lo[a] + side;
            double below = lo[a] - xk[a];
            double above = xk[a] - hi;
            double m = below > 0.0 ? below : 0.0;
            t[a] = above > m ? above : m;
        }
        double b2 = t[0] * t[0] + t[1] * t[1];
        b2 = b2 + t[2] * t[2];
        if (b2 < rcut2) return 0;
    }
    return 1;
}

typedef struct {
    const ora_tree_t *t;
    const int64_t *order;
    const double *pos, *u;
    const ora_bh_params *p;
    int use_rcut;
    float theta2_f, rcut2_f;
    double theta2_d, rcut2_d;
    const double *quad;   /* 7 per cell: S_xx, S_yy, S_zz, S_xy, S_xz, S_yz, m (p->quad only) */
} bh_ctx;

/*
 * Next term of the pseudo-particle expansion (an accuracy extension beyond
 * the paper's pseudo-particles).  A cell's particles sit at rho_i = c + d_i
 * with moments u_i; the field at r from the centre c is
 *   sum_i T(r - d_i) u_i = T(r) U - grad Phi(r) + O(d^2),
 *   Phi(r) = sum_i d_i . T(r) u_i = (3 r.S.r - m r^2) / r^5,
 * with S the symmetric part of M = sum_i d_i (x) u_i and m its trace.  The
 * force on a dipole u_k is the gradient of u_k . h, so its correction is
 * -H Phi u_k:
 *   grad Phi  = 6 S r / r^5 - 15 (r.S.r) r / r^7 + 3 m r / r^5
 *   H Phi v   = 6 S v / r^5 - 30 (r.v) S r / r^7 - 30 (S r.v) r / r^7 - 15 (r.S.r) v / r^7
 *             + 105 (r.S.r)(r.v) r / r^9 + 3 m v / r^5 - 15 m (r.v) r / r^7
 * q7 = (S_xx, S_yy, S_zz, S_xy, S_xz, S_yz, m).  Adds the corrections to h, f.
 */
static void quad_correction(const double r[3], const double q7[7], const double uk[3],
                            double h[3], double f[3])
{
    double r2 = dot3(r, r);
    double ir = 1.0 / sqrt(r2);
    double ir2 = ir * ir, ir5 = ir2 * ir2 * ir, ir7 = ir5 * ir2, ir9 = ir7 * ir2;
    double S[3][3] = {{q7[0], q7[3], q7[4]}, {q7[3], q7[1], q7[5]}, {q7[4], q7[5], q7[2]}};
    double m = q7[6];
    double Sr[3], Su[3];
    for (int a = 0; a < 3; ++a) {
        Sr[a] = S[a][0] * r[0] + S[a][1] * r[1] + S[a][2] * r[2];
        Su[a] = S[a][0] * uk[0] + S[a][1] * uk[1] + S[a][2] * uk[2];
    }
    double q = dot3(r, Sr), ru = dot3(r, uk), sru = dot3(Sr, uk);
    for (int a = 0; a < 3; ++a) {
        double gp = 6.0 * Sr[a] * ir5 - 15.0 * q * r[a] * ir7 + 3.0 * m * r[a] * ir5;
        double hp = 6.0 * Su[a] * ir5 - 30.0 * ru * Sr[a] * ir7 - 30.0 * sru * r[a] * ir7
                  - 15.0 * q * uk[a] * ir7 + 105.0 * q * ru * r[a] * ir9 + 3.0 * m * uk[a] * ir5
                  - 15.0 * m * ru * r[a] * ir7;
        h[a] -= gp;
        f[a] -= hp;
    }
}

typedef struct {
    double h[3], fd[3], fs[3], e_sr;
    double habs, fdabs, fsabs;   /* sums of the magnitudes of the terms added */
    int64_t nacc, npair, nopen, ncover;
    /* optional list of the sources in visiting order, three words each:
       (0, pbegin, pend) for an accepted cell, (1, s, s + 1) for the particle at
       sorted position s summed exactly; nsrc counts past src_cap */
    int64_t *src, nsrc, src_cap;
} bh_acc;

static void rec_src(bh_acc *acc, int64_t kind, int64_t a, int64_t b)
{
    if (acc->src && acc->nsrc < acc->src_cap) {
        acc->src[3 * acc->nsrc] = kind;
        acc->src[3 * acc->nsrc + 1] = a;
        acc->src[3 * acc->nsrc + 2] = b;
    }
    acc->nsrc++;
}

/* per-particle recursive visit, children in octant order (Sec. 3.2) */
static void bh_visit(const bh_ctx *g, int64_t k, int64_t sk, int64_t c, bh_acc *acc)
{
    const ora_tree_t *t = g->t;
    const double *xk = &g->pos[3 * k];
    const double *uk = &g->u[3 * k];
    int inside = (t->pbegin[c] <= sk && sk < t->pend[c]);
    int ok = 0;
    if (!inside) {
        if (g->p->prec != 1) {
            float xf[3], cf[3], lof[3];
            for (int a = 0; a < 3; ++a) {
                xf[a] = (float)xk[a];
                cf[a] = (float)t->cen[3 * c + a];
                lof[a] = (float)t->lo[3 * c + a];
            }
            ok = accept_f(xf, cf, (float)t->side[c], lof, g->theta2_f, g->use_rcut, g->rcut2_f);
        } else {
            ok = accept_d(xk, &t->cen[3 * c], t->side[c], &t->lo[3 * c], g->theta2_d,
                          g->use_rcut, g->rcut2_d);
        }
    }
    if (ok) {
        /* pseudo-particle: moment U, position = centre (Eq. magCenter) */
        double r[3], hp[3], fp[3];
        for (int a = 0; a < 3; ++a) r[a] = xk[a] - t->cen[3 * c + a];
        if (dot3(r, r) > 0.0) {
            ora_pair_dipole(r, uk, &t->U64[3 * c], hp, fp);
            if (g->quad) quad_correction(r, &g->quad[7 * c], uk, hp, fp);
            for (int a = 0; a < 3; ++a) { acc->h[a] += hp[a]; acc->fd[a] += fp[a]; }
            acc->habs += sqrt(dot3(hp, hp));
            acc->fdabs += sqrt(dot3(fp, fp));
        }
        acc->nacc++;
        acc->ncover += t->pend[c] - t->pbegin[c];
        rec_src(acc, 0, t->pbegin[c], t->pend[c]);
        return;
    }
    if (t->leaf[c]) {
        for (int64_t s = t->pbegin[c]; s < t->pend[c]; ++s) {
            if (s == sk) continue;
            int64_t j = g->order[s];
            double r[3], hp[3], fp[3];
            for (int a = 0; a < 3; ++a) r[a] = xk[a] - g->pos[3 * j + a];
            acc->npair++;
            rec_src(acc, 1, s, s + 1);
            if (dot3(r, r) == 0.0) continue;
            ora_pair_dipole(r, uk, &g->u[3 * j], hp, fp);
            for (int a = 0; a < 3; ++a) { acc->h[a] += hp[a]; acc->fd[a] += fp[a]; }
            acc->habs += sqrt(dot3(hp, hp));
            acc->fdabs += sqrt(dot3(fp, fp));
            if (g->use_rcut && g->p->include_sr &&
                lj_inside(xk, &g->pos[3 * j], g->p->lj_rcut, g->p->prec)) {
                double fl[3];
                acc->e_sr += 0.5 * lj_pair_inside(r, g->p->lj_eps, g->p->lj_sigma, g->p->lj_rcut, fl);
                for (int a = 0; a < 3; ++a) acc->fs[a] += fl[a];
                acc->fsabs += sqrt(dot3(fl, fl));
            }
        }
        return;
    }
    acc->nopen++;
    int64_t ch = c + 1;
    while (ch < t->skip[c]) {
        bh_visit(g, k, sk, ch, acc);
        ch = t->skip[ch];
    }
}

/*
 * Barnes-Hut field and force on every particle (or on the n_only particles
 * listed in `only`; other rows are left untouched).  Outputs are in input
 * order: h = dip_scale * h_dip, f = dip_scale * f_dip + f_sr, e_sr = half
 * the shifted LJ energy of k's pairs.  nacc / npair / nopen count accepted
 * cells, exact pairs evaluated and cells opened; ncover counts the particles
 * inside accepted cells (ncover + npair = n - 1 when every other particle is
 * reached exactly once).  habs / fabs (may be NULL) receive the sums of the
 * magnitudes of the terms that make up h and f (with the same dip_scale): the
 * scale against which the rounding of a sum with cancellation is measured.
 * Returns the cell count.
 */
int64_t ora_bh(int64_t n, const double *pos, const double *u, const ora_bh_params *p,
               const int64_t *only, int64_t n_only,
               double *h, double *f, double *e_sr, int64_t *nacc, int64_t *npair, int64_t *nopen,
               int64_t *ncover, double *habs, double *fabs_out)
{
    uint64_t *skeys = malloc(n * sizeof(uint64_t));
    int64_t *order = malloc(n * sizeof(int64_t));
    int64_t *rank = malloc(n * sizeof(int64_t));
    double root[4];
    ora_tree_t t;
    tree_build(n, pos, u, p->prec, p->leaf_max, skeys, order, root, &t);
    for (int64_t s = 0; s < n; ++s) rank[order[s]] = s;

    bh_ctx g;
    g.t = &t;
    g.order = order;
    g.pos = pos;
    g.u = u;
    g.p = p;
    g.use_rcut = (p->lj_eps != 0.0 && p->lj_rcut > 0.0);
    g.theta2_d = p->theta * p->theta;
    g.theta2_f = (float)g.theta2_d;
    g.rcut2_d = g.use_rcut ? p->lj_rcut * p->lj_rcut : 0.0;
    g.rcut2_f = (float)g.rcut2_d;
    g.quad = NULL;
    double *quad = NULL;
    if (p->quad) {
        /* S and m of every cell about its pseudo-particle position, from its particles */
        quad = calloc(7 * t.n, sizeof(double));
        for (int64_t c = 0; c < t.n; ++c) {
            double *q7 = &quad[7 * c];
            for (int64_t s = t.pbegin[c]; s < t.pend[c]; ++s) {
                int64_t j = order[s];
                double d[3];
                for (int a = 0; a < 3; ++a) d[a] = pos[3 * j + a] - t.cen[3 * c + a];
                const double *uj = &u[3 * j];
                q7[0] += d[0] * uj[0];
                q7[1] += d[1] * uj[1];
                q7[2] += d[2] * uj[2];
                q7[3] += 0.5 * (d[0] * uj[1] + d[1] * uj[0]);
                q7[4] += 0.5 * (d[0] * uj[2] + d[2] * uj[0]);
                q7[5] += 0.5 * (d[1] * uj[2] + d[2] * uj[1]);
                q7[6] += dot3(d, uj);
            }
        }
        g.quad = quad;
    }

    int64_t cnt = only ? n_only : n;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < cnt; ++q) {
        int64_t k = only ? only[q] : q;
        bh_acc acc;
        memset(&acc, 0, sizeof(acc));
        bh_visit(&g, k, rank[k], 0, &acc);
        for (int a = 0; a < 3; ++a) {
            h[3 * k + a] = p->dip_scale * acc.h[a];
            f[3 * k + a] = p->dip_scale * acc.fd[a] + acc.fs[a];
        }
        if (e_sr) e_sr[k] = acc.e_sr;
        if (nacc) nacc[k] = acc.nacc;
        if (npair) npair[k] = acc.npair;
        if (nopen) nopen[k] = acc.nopen;
        if (ncover) ncover[k] = acc.ncover;
        if (habs) habs[k] = fabs(p->dip_scale) * acc.habs;
        if (fabs_out) fabs_out[k] = fabs(p->dip_scale) * acc.fdabs + acc.fsabs;
    }
    int64_t nc = t.n;
    free(quad);
    tree_free(&t);
    free(skeys);
    free(order);
    free(rank);
    return nc;
}

/*
 * The sources of one particle (input index k) in the order the traversal of
 * ora_bh visits them: three words per source in src (at most cap sources
 * stored), (0, pbegin, pend) for a cell accepted as its pseudo-particle and
 * (1, s, s + 1) for the particle at sorted position s summed exactly; order
 * (n words) receives the sorted position -> input index map, so a source's
 * particles are order[pbegin .. pend).  Returns the number of sources (larger
 * than cap when the list did not fit).  This is ora_bh's own visit, so the
 * list shows exactly the opening decisions its field sums follow.
 */
int64_t ora_bh_sources(int64_t n, const double *pos, const double *u, const ora_bh_params *p,
                       int64_t k, int64_t *order, int64_t *src, int64_t cap)
{
    uint64_t *skeys = malloc(n * sizeof(uint64_t));
    double root[4];
    ora_tree_t t;
    tree_build(n, pos, u, p->prec, p->leaf_max, skeys, order, root, &t);
    int64_t sk = 0;
    for (int64_t s = 0; s < n; ++s)
        if (order[s] == k) sk = s;
    bh_ctx g;
    g.t = &t;
    g.order = order;
    g.pos = pos;
    g.u = u;
    g.p = p;
    g.use_rcut = (p->lj_eps != 0.0 && p->lj_rcut > 0.0);
    g.theta2_d = p->theta * p->theta;
    g.theta2_f = (float)g.theta2_d;
    g.rcut2_d = g.use_rcut ? p->lj_rcut * p->lj_rcut : 0.0;
    g.rcut2_f = (float)g.rcut2_d;
    g.quad = NULL;
    bh_acc acc;
    memset(&acc, 0, sizeof(acc));
    acc.src = src;
    acc.src_cap = cap;
    bh_visit(&g, k, sk, 0, &acc);
    tree_free(&t);
    free(skeys);
    return acc.nsrc;
}

/* ------------------------------------------------------------------------ */
/* gradient of the Barnes-Hut dipolar energy (decisions frozen)             */
/* ------------------------------------------------------------------------ */
/*
 * E = -1/2 * dip_scale * sum_m u_m . H_m with H_m = sum over m's sources s of
 * T(rho_m - x_s) w_s, T(r) = (3 r r^T - r^2 I) / r^5 (Sec. 2, Eq. h_dip), the
 * sources being the cells m accepts (x = mean position of the cell's
 * particles, w = their moment sum, Eq. magCenter) and the particles it sums
 * exactly.  Which sources m sees is decided on a reference configuration
 * pos_dec (the opening test of Sec. 3.2 is piecewise constant in the
 * positions); E and its gradient are evaluated at pos with those decisions
 * frozen, so a central difference of E that moves pos but keeps pos_dec is a
 * difference of one smooth function.
 *
 * With phi(r; a, b) = a . T(r) b (symmetric in a, b; its r-gradient is the
 * printed force f_dip):
 *   dE/du_k   = -1/2 ds [ H_k + sum over (m, s) with k in s of T(rho_m - x_s) u_m ]
 *   dE/drho_k = -1/2 ds [ F_k - sum over (m, s) with k in s of
 *                          grad phi(rho_m - x_s; u_m, w_s) / n_s ]
 * where F_k = sum_s grad phi(rho_k - x_s; u_k, w_s) and n_s is the number of
 * particles in s.  Returns E; grad_pos and grad_u are n x 3.
 * tree_centres = 0: a cell's x_s is the exact mean of its particles' current
 * positions (E is then one smooth function of pos); 1: the centre of the
 * decision tree in its own precision (as the Barnes-Hut field uses it; with
 * pos = pos_dec this differs from the exact mean by the tree precision's
 * rounding only), for comparing with a single-precision implementation.
 */
typedef struct {
    const bh_ctx *g;          /* decisions: tree of pos_dec */
    const double *pos_dec;
    const double *cc, *uc;    /* current centre and moment sum of every cell */
    double *acc;              /* this thread's source sums: 6 per cell, then 6 per particle */
    double H[3], F[3];
} grad_ctx;

static void grad_term(grad_ctx *q, int64_t m, const double *xs, const double *ws, double *sum6)
{
    const double *xm = &q->g->pos[3 * m];
    const double *um = &q->g->u[3 * m];
    double r[3], hp[3], fp[3], hr[3], fr[3];
    for (int a = 0; a < 3; ++a) r[a] = xm[a] - xs[a];
    if (dot3(r, r) == 0.0) return;
    ora_pair_dipole(r, um, ws, hp, fp);   /* field of the source at m, force on m */
    for (int a = 0; a < 3; ++a) { q->H[a] += hp[a]; q->F[a] += fp[a]; }
    ora_pair_dipole(r, ws, um, hr, fr);   /* T(r) u_m and grad phi(r; w_s, u_m) */
    for (int a = 0; a < 3; ++a) { sum6[a] += hr[a]; sum6[3 + a] += fr[a]; }
}

static void grad_visit(grad_ctx *q, int64_t m, int64_t sm, int64_t c)
{
    const bh_ctx *g = q->g;
    const ora_tree_t *t = g->t;
    const double *xd = &q->pos_dec[3 * m];
    int inside = (t->pbegin[c] <= sm && sm < t->pend[c]);
    int ok = 0;
    if (!inside) {
        if (g->p->prec != 1) {
            float xf[3], cf[3], lof[3];
            for (int a = 0; a < 3; ++a) {
                xf[a] = (float)xd[a];
                cf[a] = (float)t->cen[3 * c + a];
                lof[a] = (float)t->lo[3 * c + a];
            }
            ok = accept_f(xf, cf, (float)t->side[c], lof, g->theta2_f, g->use_rcut, g->rcut2_f);
        } else {
            ok = accept_d(xd, &t->cen[3 * c], t->side[c], &t->lo[3 * c], g->theta2_d,
                          g->use_rcut, g->rcut2_d);
        }
    }
    if (ok) {
        grad_term(q, m, &q->cc[3 * c], &q->uc[3 * c], &q->acc[6 * c]);
        return;
    }
    if (t->leaf[c]) {
        for (int64_t s = t->pbegin[c]; s < t->pend[c]; ++s) {
            if (s == sm) continue;
            int64_t j = g->order[s];
            grad_term(q, m, &g->pos[3 * j], &g->u[3 * j], &q->acc[6 * (t->n + j)]);
        }
        return;
    }
    int64_t ch = c + 1;
    while (ch < t->skip[c]) {
        grad_visit(q, m, sm, ch);
        ch = t->skip[ch];
    }
}

double ora_bh_energy_grad(int64_t n, const double *pos, const double *u, const ora_bh_params *p,
                          const double *pos_dec, int32_t tree_centres, double *grad_pos,
                          double *grad_u)
{
    if (!pos_dec) pos_dec = pos;
    uint64_t *skeys = malloc(n * sizeof(uint64_t));
    int64_t *order = malloc(n * sizeof(int64_t));
    int64_t *rank = malloc(n * sizeof(int64_t));
    double root[4];
    ora_tree_t t;
    tree_build(n, pos_dec, u, p->prec, p->leaf_max, skeys, order, root, &t);
    for (int64_t s = 0; s < n; ++s) rank[order[s]] = s;
    const int64_t nc = t.n;

    /* current geometry of every cell: plain FP64 sums over its particles */
    double *cc = calloc(3 * nc, sizeof(double));
    double *uc = calloc(3 * nc, sizeof(double));
    for (int64_t c = 0; c < nc; ++c) {
        for (int64_t s = t.pbegin[c]; s < t.pend[c]; ++s) {
            int64_t j = order[s];
            for (int a = 0; a < 3; ++a) {
                cc[3 * c + a] += pos[3 * j + a];
                uc[3 * c + a] += u[3 * j + a];
            }
        }
        double cnt = (double)(t.pend[c] - t.pbegin[c]);
        for (int a = 0; a < 3; ++a)
            cc[3 * c + a] = tree_centres ? t.cen[3 * c + a] : cc[3 * c + a] / cnt;
    }

    bh_ctx g;
    g.t = &t;
    g.order = order;
    g.pos = pos;
    g.u = u;
    g.p = p;
    g.use_rcut = (p->lj_eps != 0.0 && p->lj_rcut > 0.0);
    g.theta2_d = p->theta * p->theta;
    g.theta2_f = (float)g.theta2_d;
    g.rcut2_d = g.use_rcut ? p->lj_rcut * p->lj_rcut : 0.0;
    g.rcut2_f = (float)g.rcut2_d;
    g.quad = NULL;  /* the gradients use the paper's pseudo-particles only */

    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    const int64_t nsrc = nc + n;
    double *acc = calloc((size_t)nthr * 6 * nsrc, sizeof(double));
    double *H = calloc(3 * n, sizeof(double));
    double *F = calloc(3 * n, sizeof(double));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t m = 0; m < n; ++m) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        grad_ctx q;
        q.g = &g;
        q.pos_dec = pos_dec;
        q.cc = cc;
        q.uc = uc;
        q.acc = acc + (size_t)tid * 6 * nsrc;
        memset(q.H, 0, sizeof(q.H));
        memset(q.F, 0, sizeof(q.F));
        grad_visit(&q, m, rank[m], 0);
        for (int a = 0; a < 3; ++a) {
            H[3 * m + a] = q.H[a];
            F[3 * m + a] = q.F[a];
        }
    }
    /* source sums over the threads, in thread order */
    for (int th = 1; th < nthr; ++th)
        for (int64_t i = 0; i < 6 * nsrc; ++i) acc[i] += acc[(size_t)th * 6 * nsrc + i];

    /* push each cell's sums to its particles; particle sources to themselves */
    double *gsum = calloc(3 * n, sizeof(double));
    double *qsum = calloc(3 * n, sizeof(double));
    for (int64_t c = 0; c < nc; ++c) {
        double cnt = (double)(t.pend[c] - t.pbegin[c]);
        for (int64_t s = t.pbegin[c]; s < t.pend[c]; ++s) {
            int64_t k = order[s];
            for (int a = 0; a < 3; ++a) {
                gsum[3 * k + a] += acc[6 * c + a];
                qsum[3 * k + a] += acc[6 * c + 3 + a] / cnt;
            }
        }
    }
    for (int64_t k = 0; k < n; ++k)
        for (int a = 0; a < 3; ++a) {
            gsum[3 * k + a] += acc[6 * (nc + k) + a];
            qsum[3 * k + a] += acc[6 * (nc + k) + 3 + a];
        }
    double E = 0.0;
    const double ds = p->dip_scale;
    for (int64_t k = 0; k < n; ++k) {
        E += dot3(&u[3 * k], &H[3 * k]);
        for (int a = 0; a < 3; ++a) {
            grad_u[3 * k + a] = -0.5 * ds * (H[3 * k + a] + gsum[3 * k + a]);
            grad_pos[3 * k + a] = -0.5 * ds * (F[3 * k + a] - qsum[3 * k + a]);
        }
    }
    E *= -0.5 * ds;
    free(gsum); free(qsum); free(acc); free(H); free(F); free(cc); free(uc);
    tree_free(&t);
    free(skeys); free(order); free(rank);
    return E;
}


/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)                         */
/* ------------------------------------------------------------------------ */
/*
 * One round: multiply words 0 and 2 by the round multipliers, take high and
 * low halves, and mix with the other words and the round key.  Ten rounds;
 * the key is bumped by the Weyl constants between rounds.
 */
static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }
        philox_round(c, k);
    }
    for (int i = 0; i < 4; ++i) out[i] = c[i];
}

/*
 * Eight standard normals for particle `id` at step `step` (reading of the
 * white noise of Sec. 2): key = (seed lo, seed hi), counter = (step lo,
 * step hi, id, block) for block 0 and 1; each pair (a, b) of words gives
 * u1 = (a + 1) 2^-32 in (0, 1], u2 = b 2^-32 and, by Box-Muller,
 * z0 = sqrt(-2 ln u1) cos(2 pi u2), z1 = sqrt(-2 ln u1) sin(2 pi u2).
 */
void ora_normals(uint64_t seed, uint64_t step, uint32_t id, double z[8])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (uint32_t blk = 0; blk < 2; ++blk) {
        uint32_t ctr[4] = {(uint32_t)step, (uint32_t)(step >> 32), id, blk};
        uint32_t w[4];
        ora_philox4x32_10(ctr, key, w);
        for (int p = 0; p < 2; ++p) {
            double u1 = ((double)w[2 * p] + 1.0) * 0x1p-32;
            double u2 = (double)w[2 * p + 1] * 0x1p-32;
            double rad = sqrt(-2.0 * log(u1));
            z[4 * blk + 2 * p] = rad * cos(2.0 * M_PI * u2);
            z[4 * blk + 2 * p + 1] = rad * sin(2.0 * M_PI * u2);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* walls and the Euler-Maruyama step                                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    double dt;
    double gamma_t, gamma_r;
    double inertia;        /* 2/5 in reduced units (Sec. 2) */
    double kT;
    double rot_noise;      /* fluctuation-dissipation: 2 */
    double h_ext[3];
    double box_lo[3], box_hi[3];
    int32_t walls;
    int32_t literal;       /* 1: the printed angle equations (see ora_em_step) */
    double wall_eps;
    uint64_t seed;
} ora_dyn;

#define ORA_WALL_SIGMA 0.5
#define ORA_WALL_WMIN 0.01

/*
 * Wall force along one axis ("LJ of the same type", Sec. 2): with w the
 * distance from the centre to the plane, sigma_w = 1/2 and the force cut
 * where it vanishes (w = sigma_w), F = 24 eps / w [(s/w)^12 - (s/w)^6],
 * pushing away from the plane; w is clamped below at 0.01.  Energy
 * 2 eps (s/w)^12 - 4 eps (s/w)^6 + 2 eps (zero at the cut).
 */
static double wall_f(double w, double eps, double *e)
{
    if (!(w < ORA_WALL_SIGMA)) { *e = 0.0; return 0.0; }
    if (w < ORA_WALL_WMIN) w = ORA_WALL_WMIN;
    double s = ORA_WALL_SIGMA / w;
    double s2 = s * s;
    double s6 = s2 * s2 * s2;
    *e = 2.0 * eps * s6 * s6 - 4.0 * eps * s6 + 2.0 * eps;
    return 24.0 * eps * (s6 * s6 - s6) / w;
}

/* wall force and energy on one particle; planes at box_lo - 1/2 and box_hi + 1/2 */
void ora_wall(const double x[3], const ora_dyn *d, double fw[3], double *ew)
{
    *ew = 0.0;
    fw[0] = fw[1] = fw[2] = 0.0;
    if (!d->walls) return;
    for (int a = 0; a < 3; ++a) {
        double e1, e2;
        fw[a] += wall_f(x[a] - (d->box_lo[a] - 0.5), d->wall_eps, &e1);
        fw[a] -= wall_f((d->box_hi[a] + 0.5) - x[a], d->wall_eps, &e2);
        *ew += e1 + e2;
    }
}

/*
 * One explicit Euler-Maruyama step (Sec. 4, dt = 1e-3) of the reduced
 * Langevin equations of Sec. 2, translational part as printed (unit reduced
 * mass) and rotational part in vector form (reading of the garbled angle
 * equations): with h = h_dip + h_ext and f = f_int + f_wall,
 *   x' = x + dt v
 *   v' = v + dt (f - G_t v) + sqrt(2 G_t kT dt) xi_t
 *   w' = w + dt (u x h - G_r w) / I + sqrt(c_r G_r kT dt) / I xi_r
 *   u' = (u + dt w x u) / |u + dt w x u|
 * all right-hand sides from the step-n state; xi_t = normals 0..2 and
 * xi_r = normals 3..5 of (seed, step, id).  Arrays are n x 3, updated in
 * place.
 *
 * With d->literal = 1 the rotation follows the printed reduced angle
 * equations instead (Sec. 2, reduced Eqs. for theta and phi, as printed):
 * theta = acos(u_z), phi = atan2(u_y, u_x), the rates (theta', phi') are kept
 * in w_x, w_y (w_z = 0), and
 *   theta'' I = (u_x h_y - u_y h_x) - G_r theta' + noise
 *   phi''   I = -(u_y h_z - u_z h_y) sin phi + (u_z h_x - u_x h_z) cos phi - G_r phi' + noise
 * stepped like the vector form (angles by their rates, rates by the torques,
 * all from the step-n state, noise normals 3 and 4), then
 * u = (sin theta cos phi, sin theta sin phi, cos theta).  Kept to document
 * that these equations do not relax toward the Boltzmann distribution (a
 * field along z exerts no torque on theta).
 */
void ora_em_step(int64_t n, double *pos, double *vel, double *u, double *om,
                 const int64_t *ids, const double *hdip, const double *fint,
                 const ora_dyn *d, uint64_t step)
{
    double st = sqrt(2.0 * d->gamma_t * d->kT * d->dt);
    double sr = sqrt(d->rot_noise * d->gamma_r * d->kT * d->dt) / d->inertia;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        double *x = &pos[3 * k], *v = &vel[3 * k], *uu = &u[3 * k], *w = &om[3 * k];
        double h[3], f[3], fw[3], ew, z[8];
        ora_wall(x, d, fw, &ew);
        for (int a = 0; a < 3; ++a) {
            h[a] = hdip[3 * k + a] + d->h_ext[a];
            f[a] = fint[3 * k + a] + fw[a];
        }
        ora_normals(d->seed, step, (uint32_t)ids[k], z);
        double tq[3] = {uu[1] * h[2] - uu[2] * h[1], uu[2] * h[0] - uu[0] * h[2],
                        uu[0] * h[1] - uu[1] * h[0]};
        double wxu[3] = {w[1] * uu[2] - w[2] * uu[1], w[2] * uu[0] - w[0] * uu[2],
                         w[0] * uu[1] - w[1] * uu[0]};
        double xn[3], vn[3], wn[3], un[3];
        for (int a = 0; a < 3; ++a) {
            xn[a] = x[a] + d->dt * v[a];
            vn[a] = v[a] + d->dt * (f[a] - d->gamma_t * v[a]) + st * z[a];
            wn[a] = w[a] + d->dt * (tq[a] - d->gamma_r * w[a]) / d->inertia + sr * z[3 + a];
            un[a] = uu[a] + d->dt * wxu[a];
        }
        double nrm = sqrt(dot3(un, un));
        for (int a = 0; a < 3; ++a) un[a] /= nrm;
        if (d->literal) {
            double uz = uu[2] < -1.0 ? -1.0 : (uu[2] > 1.0 ? 1.0 : uu[2]);
            double th = acos(uz), ph = atan2(uu[1], uu[0]);
            double tt = uu[0] * h[1] - uu[1] * h[0];
            double tp = -(uu[1] * h[2] - uu[2] * h[1]) * sin(ph)
                        + (uu[2] * h[0] - uu[0] * h[2]) * cos(ph);
            double th2 = th + d->dt * w[0], ph2 = ph + d->dt * w[1];
            wn[0] = w[0] + d->dt * (tt - d->gamma_r * w[0]) / d->inertia + sr * z[3];
            wn[1] = w[1] + d->dt * (tp - d->gamma_r * w[1]) / d->inertia + sr * z[4];
            wn[2] = 0.0;
            un[0] = sin(th2) * cos(ph2);
            un[1] = sin(th2) * sin(ph2);
            un[2] = cos(th2);
        }
        for (int a = 0; a < 3; ++a) {
            x[a] = xn[a];
            v[a] = vn[a];
            w[a] = wn[a];
            uu[a] = un[a];
        }
    }
}

/*
 * Observables (Sec. 5) and energies, FP64:
 * out[0] e_dip = -1/2 sum u.h_dip      out[1] e_zeeman = -sum u.h_ext
 * out[2] e_sr  = sum e_sr[k]           out[3] e_wall
 * out[4] e_kin_t = 1/2 sum v^2         out[5] e_kin_r = I/2 sum w^2
 * out[6..8] <u> = (1/N) sum u          out[9] <h_dip_z> = (1/N) sum h_dip_z
 */
void ora_energy(int64_t n, const double *pos, const double *vel, const double *u,
                const double *om, const double *hdip, const double *e_sr,
                const ora_dyn *d, double out[10])
{
    memset(out, 0, 10 * sizeof(double));
    for (int64_t k = 0; k < n; ++k) {
        const double *uu = &u[3 * k];
        double fw[3], ew;
        ora_wall(&pos[3 * k], d, fw, &ew);
        out[0] += -0.5 * dot3(uu, &hdip[3 * k]);
        out[1] += -dot3(uu, d->h_ext);
        out[2] += e_sr ? e_sr[k] : 0.0;
        out[3] += ew;
        out[4] += 0.5 * dot3(&vel[3 * k], &vel[3 * k]);
        out[5] += 0.5 * d->inertia * dot3(&om[3 * k], &om[3 * k]);
        for (int a = 0; a < 3; ++a) out[6 + a] += uu[a];
        out[9] += hdip[3 * k + 2];
    }
    for (int a = 0; a < 3; ++a) out[6 + a] /= (double)n;
    out[9] /= (double)n;
}

/* ------------------------------------------------------------------------ */
/* reverse mode: field and force VJP, Euler-Maruyama adjoint, d<M_z>/dh      */
/* ------------------------------------------------------------------------ */
/*
 * Hessian of phi(r; a, b) = a . T(r) b applied to v, i.e. the derivative along
 * v of the printed force 3[a(b.r) + b(a.r) + r(a.b)]/r^5 - 15 r(a.r)(b.r)/r^7:
 *   3[(a.v) b + (b.v) a + (a.b) v]/r^5
 *   - 15 [r((a.v)(b.r) + (b.v)(a.r) + (r.v)(a.b)) + v (a.r)(b.r) + (r.v)(a (b.r) + b (a.r))]/r^7
 *   + 105 r (r.v)(a.r)(b.r)/r^9
 */
static void phi_hess(const double r[3], const double a[3], const double b[3], const double v[3],
                     double out[3])
{
    double r2 = dot3(r, r);
    double ir = 1.0 / sqrt(r2);
    double ir2 = ir * ir;
    double ir5 = ir2 * ir2 * ir;
    double ir7 = ir5 * ir2;
    double ir9 = ir7 * ir2;
    double ar = dot3(a, r), br = dot3(b, r), rv = dot3(r, v);
    double av = dot3(a, v), bv = dot3(b, v), ab = dot3(a, b);
    for (int c = 0; c < 3; ++c)
        out[c] = 3.0 * (av * b[c] + bv * a[c] + ab * v[c]) * ir5
               - 15.0 * (r[c] * (av * br + bv * ar + rv * ab) + v[c] * ar * br
                         + rv * (a[c] * br + b[c] * ar)) * ir7
               + 105.0 * r[c] * rv * ar * br * ir9;
}

typedef struct {
    const bh_ctx *g;
    const double *pos_dec;
    const double *cc, *uc;        /* current centre and moment sum of every cell */
    const double *abar, *bbar;    /* cotangents of h and f, n x 3 */
    double *acc;                  /* this thread's source sums: dL/dw_s, dL/dx_s (6 per source) */
    int lj;
    double hk[3], fk[3], dx[3], du[3];
} vjp_ctx;

/*
 * One interaction of target m with source s (position xs, moment sum ws),
 * r = rho_m - xs, for L = sum_m abar_m . h_m + bbar_m . f_m with
 * h_m += ds T(r) ws and f_m += ds grad phi(r; u_m, ws):
 *   dL/du_m  += ds grad phi(r; bbar_m, ws)
 *   dL/drho_m += ds [grad phi(r; abar_m, ws) + H phi(r; u_m, ws) bbar_m] = g
 *   dL/dws   += ds [T(r) abar_m + grad phi(r; bbar_m, u_m)]
 *   dL/dxs   -= g
 * (the r-Jacobian of T(r) w is symmetric, so its product with a vector is
 * grad phi of that vector).
 */
static void vjp_term(vjp_ctx *q, int64_t m, const double *xs, const double *ws, double *src6)
{
    const bh_ctx *g = q->g;
    const double ds = g->p->dip_scale;
    const double *xm = &g->pos[3 * m], *um = &g->u[3 * m];
    const double *a = &q->abar[3 * m], *b = &q->bbar[3 * m];
    double r[3], hp[3], fp[3], t1[3], t2[3], t3[3], t4[3], t5[3], dummy[3];
    for (int c = 0; c < 3; ++c) r[c] = xm[c] - xs[c];
    if (dot3(r, r) == 0.0) return;
    ora_pair_dipole(r, um, ws, hp, fp);    /* forward: T(r) ws, grad phi(r; u_m, ws) */
    ora_pair_dipole(r, b, ws, dummy, t1);  /* grad phi(r; bbar, ws) */
    ora_pair_dipole(r, a, ws, dummy, t2);  /* grad phi(r; abar, ws) */
    phi_hess(r, um, ws, b, t3);
    ora_pair_dipole(r, um, a, t4, dummy);  /* T(r) abar */
    ora_pair_dipole(r, b, um, dummy, t5);  /* grad phi(r; bbar, u_m) */
    for (int c = 0; c < 3; ++c) {
        q->hk[c] += ds * hp[c];
        q->fk[c] += ds * fp[c];
        q->du[c] += ds * t1[c];
        double gc = ds * (t2[c] + t3[c]);
        q->dx[c] += gc;
        src6[c] += ds * (t4[c] + t5[c]);
        src6[3 + c] -= gc;
    }
}

/*
 * LJ pair (Eq. LJ) of target m with particle j inside the cut: f_m += c r,
 * c = 24 eps (s^12 - s^6) / r^2 with s = sigma / r.  The pair enters
 * L through bbar_m . c r + bbar_j . c (-r) = c (bbar_m - bbar_j) . r, whose
 * derivative in rho_m is c db + 2 c'(r^2) (db . r) r, db = bbar_m - bbar_j,
 * c' = dc / d(r^2) = 24 eps (-7 s^12 + 4 s^6) / r^4.  Every pair inside the cut
 * is summed exactly by both of its particles, so each adds its own derivative.
 */
static void vjp_lj(vjp_ctx *q, int64_t m, int64_t j)
{
    const bh_ctx *g = q->g;
    const double *xm = &g->pos[3 * m], *xj = &g->pos[3 * j];
    double r[3], db[3];
    for (int c = 0; c < 3; ++c) {
        r[c] = xm[c] - xj[c];
        db[c] = q->bbar[3 * m + c] - q->bbar[3 * j + c];
    }
    double r2 = dot3(r, r);
    double s2 = g->p->lj_sigma * g->p->lj_sigma / r2;
    double s6 = s2 * s2 * s2;
    double eps24 = 24.0 * g->p->lj_eps;
    double cc = eps24 * (s6 * s6 - s6) / r2;
    double dc = eps24 * (-7.0 * s6 * s6 + 4.0 * s6) / (r2 * r2);
    double dbr = dot3(db, r);
    for (int c = 0; c < 3; ++c) {
        q->fk[c] += cc * r[c];
        q->dx[c] += cc * db[c] + 2.0 * dc * dbr * r[c];
    }
}

static void vjp_visit(vjp_ctx *q, int64_t m, int64_t sm, int64_t c)
{
    const bh_ctx *g = q->g;
    const ora_tree_t *t = g->t;
    const double *xd = &q->pos_dec[3 * m];
    int inside = (t->pbegin[c] <= sm && sm < t->pend[c]);
    int ok = 0;
    if (!inside) {
        if (g->p->prec != 1) {
            float xf[3], cf[3], lof[3];
            for (int a = 0; a < 3; ++a) {
                xf[a] = (float)xd[a];
                cf[a] = (float)t->cen[3 * c + a];
                lof[a] = (float)t->lo[3 * c + a];
            }
            ok = accept_f(xf, cf, (float)t->side[c], lof, g->theta2_f, g->use_rcut, g->rcut2_f);
        } else {
            ok = accept_d(xd, &t->cen[3 * c], t->side[c], &t->lo[3 * c], g->theta2_d,
                          g->use_rcut, g->rcut2_d);
        }
    }
    if (ok) {
        vjp_term(q, m, &q->cc[3 * c], &q->uc[3 * c], &q->acc[6 * c]);
        return;
    }
    if (t->leaf[c]) {
        for (int64_t s = t->pbegin[c]; s < t->pend[c]; ++s) {
            if (s == sm) continue;
            int64_t j = g->order[s];
            vjp_term(q, m, &g->pos[3 * j], &g->u[3 * j], &q->acc[6 * (t->n + j)]);
            if (q->lj && lj_inside(&g->pos[3 * m], &g->pos[3 * j], g->p->lj_rcut, g->p->prec))
                vjp_lj(q, m, j);
        }
        return;
    }
    int64_t ch = c + 1;
    while (ch < t->skip[c]) {
        vjp_visit(q, m, sm, ch);
        ch = t->skip[ch];
    }
}

/*
 * Vector-Jacobian product of the Barnes-Hut field and force (Sec. 3.2, the
 * decisions of pos_dec frozen, as ora_bh_energy_grad): for
 * L = sum_m abar_m . h_m + bbar_m . f_m, with h the dipolar field and f the
 * dipolar force plus, when p->include_sr, the LJ force, writes dL/dpos and
 * dL/du (n x 3).  h_out and f_out (may be NULL) receive the field and force
 * of the same frozen evaluation.
 */
void ora_bh_vjp(int64_t n, const double *pos, const double *u, const ora_bh_params *p,
                const double *pos_dec, int32_t tree_centres, const double *abar,
                const double *bbar, double *dpos, double *du, double *h_out, double *f_out)
{
    if (!pos_dec) pos_dec = pos;
    uint64_t *skeys = malloc(n * sizeof(uint64_t));
    int64_t *order = malloc(n * sizeof(int64_t));
    int64_t *rank = malloc(n * sizeof(int64_t));
    double root[4];
    ora_tree_t t;
    tree_build(n, pos_dec, u, p->prec, p->leaf_max, skeys, order, root, &t);
    for (int64_t s = 0; s < n; ++s) rank[order[s]] = s;
    const int64_t nc = t.n;
    double *cc = calloc(3 * nc, sizeof(double));
    double *uc = calloc(3 * nc, sizeof(double));
    for (int64_t c = 0; c < nc; ++c) {
        for (int64_t s = t.pbegin[c]; s < t.pend[c]; ++s) {
            int64_t j = order[s];
            for (int a = 0; a < 3; ++a) {
                cc[3 * c + a] += pos[3 * j + a];
                uc[3 * c + a] += u[3 * j + a];
            }
        }
        double cnt = (double)(t.pend[c] - t.pbegin[c]);
        for (int a = 0; a < 3; ++a)
            cc[3 * c + a] = tree_centres ? t.cen[3 * c + a] : cc[3 * c + a] / cnt;
    }
    bh_ctx g;
    g.t = &t;
    g.order = order;
    g.pos = pos;
    g.u = u;
    g.p = p;
    g.use_rcut = (p->lj_eps != 0.0 && p->lj_rcut > 0.0);
    g.theta2_d = p->theta * p->theta;
    g.theta2_f = (float)g.theta2_d;
    g.rcut2_d = g.use_rcut ? p->lj_rcut * p->lj_rcut : 0.0;
    g.rcut2_f = (float)g.rcut2_d;
    g.quad = NULL;  /* the gradients use the paper's pseudo-particles only */
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    const int64_t nsrc = nc + n;
    double *acc = calloc((size_t)nthr * 6 * nsrc, sizeof(double));
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t m = 0; m < n; ++m) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        vjp_ctx q;
        memset(&q, 0, sizeof(q));
        q.g = &g;
        q.pos_dec = pos_dec;
        q.cc = cc;
        q.uc = uc;
        q.abar = abar;
        q.bbar = bbar;
        q.acc = acc + (size_t)tid * 6 * nsrc;
        q.lj = g.use_rcut && p->include_sr;
        vjp_visit(&q, m, rank[m], 0);
        for (int a = 0; a < 3; ++a) {
            dpos[3 * m + a] = q.dx[a];
            du[3 * m + a] = q.du[a];
            if (h_out) h_out[3 * m + a] = q.hk[a];
            if (f_out) f_out[3 * m + a] = q.fk[a];
        }
    }
    for (int th = 1; th < nthr; ++th)
        for (int64_t i = 0; i < 6 * nsrc; ++i) acc[i] += acc[(size_t)th * 6 * nsrc + i];
    for (int64_t c = 0; c < nc; ++c) {
        double cnt = (double)(t.pend[c] - t.pbegin[c]);
        for (int64_t s = t.pbegin[c]; s < t.pend[c]; ++s) {
            int64_t k = order[s];
            for (int a = 0; a < 3; ++a) {
                du[3 * k + a] += acc[6 * c + a];
                dpos[3 * k + a] += acc[6 * c + 3 + a] / cnt;
            }
        }
    }
    for (int64_t k = 0; k < n; ++k)
        for (int a = 0; a < 3; ++a) {
            du[3 * k + a] += acc[6 * (nc + k) + a];
            dpos[3 * k + a] += acc[6 * (nc + k) + 3 + a];
        }
    free(acc); free(cc); free(uc);
    tree_free(&t);
    free(skeys); free(order); free(rank);
}

/* dF/dw of the wall force F(w) = 24 eps (s^12 - s^6) / w, s = sigma_w / w; zero
   where the force is cut (w >= sigma_w) or w is clamped */
static double wall_df(double w, double eps)
{
    if (!(w < ORA_WALL_SIGMA)) return 0.0;
    if (w < ORA_WALL_WMIN) return 0.0;
    double s = ORA_WALL_SIGMA / w;
    double s2 = s * s;
    double s6 = s2 * s2 * s2;
    return 24.0 * eps * (-13.0 * s6 * s6 + 7.0 * s6) / (w * w);
}

/*
 * Adjoint of one Euler-Maruyama step of ora_em_step for one particle.
 * In: the step-n state (x, v, u, w), the dipolar field hdip and interaction
 * force fint of that state, and the adjoints of the step's outputs in
 * (xb, vb, ub, wb), which are replaced by the adjoints of its inputs
 * (without the field's and force's own dependence on x and u).  Out: the
 * cotangents of hdip (abar) and fint (bbar), and the cotangent of the applied
 * field accumulated into hb[3].
 *   u' = a / |a|, a = u + dt w x u:   abar_a = (ub' - u'(u'.ub')) / |a|
 *       ub = abar_a - dt w x abar_a;  wb = dt u x abar_a
 *   w' = w + dt (u x h - Gr w) / I:   wb += (1 - dt Gr / I) wb';  ub += dt/I h x wb'
 *       hbar = dt/I wb' x u (cotangent of h = hdip + h_ext)
 *   v' = v + dt (f - Gt v):          vb = (1 - dt Gt) vb';  fbar = dt vb'
 *   x' = x + dt v:                    xb = xb' + walls' dF/dx fbar;  vb += dt xb'
 */
static void em_step_vjp1(const double x[3], const double u[3], const double w[3],
                         const double hdip[3], const ora_dyn *d, double xb[3], double vb[3],
                         double ub[3], double wb[3], double abar[3], double bbar[3], double hb[3])
{
    const double dt = d->dt;
    double h[3], a[3], wxu[3], un[3];
    for (int c = 0; c < 3; ++c) h[c] = hdip[c] + d->h_ext[c];
    wxu[0] = w[1] * u[2] - w[2] * u[1];
    wxu[1] = w[2] * u[0] - w[0] * u[2];
    wxu[2] = w[0] * u[1] - w[1] * u[0];
    for (int c = 0; c < 3; ++c) a[c] = u[c] + dt * wxu[c];
    double l = sqrt(dot3(a, a));
    for (int c = 0; c < 3; ++c) un[c] = a[c] / l;
    double p = dot3(un, ub);
    double aa[3];
    for (int c = 0; c < 3; ++c) aa[c] = (ub[c] - un[c] * p) / l;
    double nub[3], nwb[3], nvb[3], nxb[3];
    /* ub = aa - dt w x aa; wb = dt u x aa */
    nub[0] = aa[0] - dt * (w[1] * aa[2] - w[2] * aa[1]);
    nub[1] = aa[1] - dt * (w[2] * aa[0] - w[0] * aa[2]);
    nub[2] = aa[2] - dt * (w[0] * aa[1] - w[1] * aa[0]);
    nwb[0] = dt * (u[1] * aa[2] - u[2] * aa[1]);
    nwb[1] = dt * (u[2] * aa[0] - u[0] * aa[2]);
    nwb[2] = dt * (u[0] * aa[1] - u[1] * aa[0]);
    const double ci = dt / d->inertia;
    for (int c = 0; c < 3; ++c) nwb[c] += (1.0 - ci * d->gamma_r) * wb[c];
    /* ub += dt/I h x wb';  hbar = dt/I wb' x u */
    nub[0] += ci * (h[1] * wb[2] - h[2] * wb[1]);
    nub[1] += ci * (h[2] * wb[0] - h[0] * wb[2]);
    nub[2] += ci * (h[0] * wb[1] - h[1] * wb[0]);
    abar[0] = ci * (wb[1] * u[2] - wb[2] * u[1]);
    abar[1] = ci * (wb[2] * u[0] - wb[0] * u[2]);
    abar[2] = ci * (wb[0] * u[1] - wb[1] * u[0]);
    for (int c = 0; c < 3; ++c) {
        hb[c] += abar[c];
        nvb[c] = (1.0 - dt * d->gamma_t) * vb[c] + dt * xb[c];
        bbar[c] = dt * vb[c];
        nxb[c] = xb[c];
    }
    if (d->walls)
        for (int c = 0; c < 3; ++c) {
            double dfl = wall_df(x[c] - (d->box_lo[c] - 0.5), d->wall_eps);
            double dfu = wall_df((d->box_hi[c] + 0.5) - x[c], d->wall_eps);
            nxb[c] += bbar[c] * (dfl + dfu);
        }
    for (int c = 0; c < 3; ++c) {
        xb[c] = nxb[c];
        vb[c] = nvb[c];
        ub[c] = nub[c];
        wb[c] = nwb[c];
    }
}

/*
 * Sensitivity of the mean magnetisation to the applied field (Sec. 5): runs
 * nsteps steps of ora_em_step from the given state (particle ids 0..n-1,
 * Philox steps 0..nsteps-1) with the Barnes-Hut (or, at theta = 0, exact)
 * field and force of p, and returns
 *   Mz = 1/nsteps sum_{t=1..nsteps} 1/n sum_k u_z,k(t)
 * with its derivative with respect to h_ext in dmz_dh[3], by reverse mode
 * through every step (the decisions of each step frozen; noise is additive
 * and keyed by (seed, step, id), so it does not depend on h_ext).  The input
 * state is left unchanged.  Vector rotor form only (d->literal = 0).
 */
double ora_mz_grad(int64_t n, const double *pos0, const double *vel0, const double *u0,
                   const double *om0, const ora_dyn *d, const ora_bh_params *p, int64_t nsteps,
                   double dmz_dh[3])
{
    const size_t sz = 3 * (size_t)n;
    double *X = malloc(sizeof(double) * sz * (nsteps + 1));
    double *V = malloc(sizeof(double) * sz * (nsteps + 1));
    double *U = malloc(sizeof(double) * sz * (nsteps + 1));
    double *W = malloc(sizeof(double) * sz * (nsteps + 1));
    double *Hd = malloc(sizeof(double) * sz * (nsteps > 0 ? nsteps : 1));
    int64_t *ids = malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    for (int64_t k = 0; k < n; ++k) ids[k] = k;
    memcpy(X, pos0, sizeof(double) * sz);
    memcpy(V, vel0, sizeof(double) * sz);
    memcpy(U, u0, sizeof(double) * sz);
    memcpy(W, om0, sizeof(double) * sz);
    double *f = malloc(sizeof(double) * sz);
    double *esr = malloc(sizeof(double) * (n > 0 ? n : 1));
    double mz = 0.0;
    for (int64_t s = 0; s < nsteps; ++s) {
        double *x = X + sz * s, *v = V + sz * s, *u = U + sz * s, *w = W + sz * s;
        double *h = Hd + sz * s;
        ora_bh(n, x, u, p, NULL, 0, h, f, esr, NULL, NULL, NULL, NULL, NULL, NULL);
        memcpy(x + sz, x, sizeof(double) * sz);
        memcpy(v + sz, v, sizeof(double) * sz);
        memcpy(u + sz, u, sizeof(double) * sz);
        memcpy(w + sz, w, sizeof(double) * sz);
        ora_em_step(n, x + sz, v + sz, u + sz, w + sz, ids, h, f, d, (uint64_t)s);
        double m = 0.0;
        for (int64_t k = 0; k < n; ++k) m += (u + sz)[3 * k + 2];
        mz += m / (double)n;
    }
    mz /= (double)(nsteps > 0 ? nsteps : 1);

    double *xb = calloc(sz, sizeof(double)), *vb = calloc(sz, sizeof(double));
    double *ub = calloc(sz, sizeof(double)), *wb = calloc(sz, sizeof(double));
    double *ab = calloc(sz, sizeof(double)), *bb = calloc(sz, sizeof(double));
    double *dx = calloc(sz, sizeof(double)), *du = calloc(sz, sizeof(double));
    double hb[3] = {0.0, 0.0, 0.0};
    const double w_obs = 1.0 / ((double)n * (double)(nsteps > 0 ? nsteps : 1));
    for (int64_t s = nsteps - 1; s >= 0; --s) {
        for (int64_t k = 0; k < n; ++k) ub[3 * k + 2] += w_obs;  /* M_z of state s + 1 */
        const double *x = X + sz * s, *u = U + sz * s, *w = W + sz * s, *h = Hd + sz * s;
        for (int64_t k = 0; k < n; ++k)
            em_step_vjp1(&x[3 * k], &u[3 * k], &w[3 * k], &h[3 * k], d, &xb[3 * k], &vb[3 * k],
                         &ub[3 * k], &wb[3 * k], &ab[3 * k], &bb[3 * k], hb);
        ora_bh_vjp(n, x, u, p, NULL, 1, ab, bb, dx, du, NULL, NULL);
        for (size_t i = 0; i < sz; ++i) {
            xb[i] += dx[i];
            ub[i] += du[i];
        }
    }
    for (int c = 0; c < 3; ++c) dmz_dh[c] = hb[c];
    free(X); free(V); free(U); free(W); free(Hd); free(ids); free(f); free(esr);
    free(xb); free(vb); free(ub); free(wb); free(ab); free(bb); free(dx); free(du);
    return mz;
}
