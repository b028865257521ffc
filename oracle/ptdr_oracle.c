/*
 * Plain CPU FP64 oracle for the Pauli decomposition of Koska, Baboulin and
 * Gazda, "A tree-approach Pauli decomposition algorithm with application to
 * quantum computing" (arXiv 2403.11644).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path links,
 * loads or calls this file; only the tests, the package smoke check and the
 * CPU-baseline leg of the benchmark do.  It shares no code, header, table or
 * helper with the CUDA path.
 *
 * Everything is double precision (double _Complex) with Neumaier-compensated
 * sums.  The paper fixes no precision; it stores complex doubles (Sec. V.C.1).
 *
 * Conventions (the paper's PauliComposer notation, Sec. II.B):
 *   P = sigma_{n-1} (x) ... (x) sigma_0; qubit l <-> bit l of a row/column
 *   index (rightmost tensor factor = least significant bit).
 *   Each Pauli operator is labelled by two n-bit masks (x, z):
 *     x_l = d(sigma_l)  (1 for X and Y, the paper's diagonality function),
 *     z_l = 1 for Y and Z.
 *   The coefficient array is C[x * 2^n + z] = c_P = 2^-n tr(P A)   (Sec. II.A)
 *   A is row-major: A[r * 2^n + c].
 *
 * Functions:
 *   oracle_brute     explicit Kronecker products of the 2x2 tables, dense
 *                    trace (the straightforward method of Sec. II.A), n <= 6.
 *   oracle_direct    the O(2^n) sparse trace per coefficient (Sec. II.A,
 *                    "first optimization of the trace computation"), using
 *                    one nonzero per row at column j XOR x with value
 *                    i^{|x&z|} (-1)^{|z & (j XOR x)|}  (pinned by brute).
 *   oracle_tree      Algorithms 1-4 of Sec. III (Pauli tree, update rules
 *                    for I/X/Y/Z, compute_coeff at the leaves), with the
 *                    forest split of Sec. V.B over OpenMP threads.
 *   oracle_compose   the inverse map A = sum_P c_P P (Sec. II.A), direct.
 *   oracle_compose_fwht  the same inverse map for large n: per mask x, phase,
 *                    textbook FWHT over z, XOR-scatter.  Validated against
 *                    oracle_compose.
 *   oracle_fwht      auxiliary full check for large n: per mask x, gather the
 *                    XOR-diagonal, textbook fast Walsh-Hadamard transform,
 *                    phase and scale.  Validated against the three above.
 *   oracle_band_*    band storage (Sec. IV.A): direct formula restricted to a
 *                    mask list, a dense-gather FWHT check for large n, and a
 *                    brute-force enumeration of the masks a band can reach.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cdbl;

/* ------------------------------------------------------------------ */
/* Compensated (Neumaier) complex accumulator.                          */
/* ------------------------------------------------------------------ */
typedef struct {
    double re, im, cre, cim;
} nsum;

static void nsum_init(nsum *s) { s->re = s->im = s->cre = s->cim = 0.0; }

static void nsum_add1(double *sum, double *comp, double v)
{
    double t = *sum + v;
    if (fabs(*sum) >= fabs(v))
        *comp += (*sum - t) + v;
    else
        *comp += (v - t) + *sum;
    *sum = t;
}

static void nsum_add(nsum *s, cdbl v)
{
    nsum_add1(&s->re, &s->cre, creal(v));
    nsum_add1(&s->im, &s->cim, cimag(v));
}

static cdbl nsum_value(const nsum *s) { return (s->re + s->cre) + I * (s->im + s->cim); }

static int popc(uint64_t v) { return __builtin_popcountll(v); }

/* i^p for an integer p >= 0. */
static cdbl ipow(int p)
{
    switch (p & 3) {
    case 0: return 1.0;
    case 1: return I;
    case 2: return -1.0;
    default: return -I;
    }
}

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* ------------------------------------------------------------------ */
/* Pauli matrices, Sec. I.  Labels follow the tree order I, X, Y, Z.   */
/* ------------------------------------------------------------------ */
enum { LAB_I = 0, LAB_X = 1, LAB_Y = 2, LAB_Z = 3 };

static void pauli2x2(int lab, cdbl m[2][2])
{
    switch (lab) {
    case LAB_I: m[0][0] = 1; m[0][1] = 0; m[1][0] = 0; m[1][1] = 1; break;
    case LAB_X: m[0][0] = 0; m[0][1] = 1; m[1][0] = 1; m[1][1] = 0; break;
    case LAB_Y: m[0][0] = 0; m[0][1] = -I; m[1][0] = I; m[1][1] = 0; break;
    default:    m[0][0] = 1; m[0][1] = 0; m[1][0] = 0; m[1][1] = -1; break;
    }
}

/* d(sigma) of Sec. II.B: 1 for X and Y. */
static int lab_d(int lab) { return lab == LAB_X || lab == LAB_Y; }
/* second mask bit: 1 for Y and Z. */
static int lab_z(int lab) { return lab == LAB_Y || lab == LAB_Z; }

/* ------------------------------------------------------------------ */
/* Straightforward method: build each operator densely by Kronecker     */
/* products, then take tr(P A)/2^n (Sec. II.A).  O(16^n); n <= 6.       */
/* ------------------------------------------------------------------ */
int oracle_brute(int n, const cdbl *A, cdbl *C)
{
    if (n < 1 || n > 6) return 1;
    const uint64_t N = 1ull << n;
    const uint64_t NP = N * N; /* 4^n operators */
    const double scale = ldexp(1.0, -n);
    int rc = 0;
#pragma omp parallel
    {
        cdbl *M = malloc(sizeof(cdbl) * NP);
        cdbl *T = malloc(sizeof(cdbl) * NP);
        int labs[6];
        if (!M || !T) {
#pragma omp atomic write
            rc = 2;
        }
#pragma omp for schedule(dynamic, 16)
        for (uint64_t code = 0; code < NP; ++code) {
            if (!M || !T) continue;
            /* base-4 digit l of code = label of qubit l */
            uint64_t c = code;
            uint64_t x = 0, z = 0;
            for (int l = 0; l < n; ++l) {
                labs[l] = (int)(c & 3);
                c >>= 2;
                x |= (uint64_t)lab_d(labs[l]) << l;
                z |= (uint64_t)lab_z(labs[l]) << l;
            }
            /* P = sigma_{n-1} (x) ... (x) sigma_0, built left to right. */
            uint64_t dim = 1;
            M[0] = 1.0;
            for (int l = n - 1; l >= 0; --l) {
                cdbl s[2][2];
                pauli2x2(labs[l], s);
                uint64_t nd = dim * 2;
                for (uint64_t i = 0; i < dim; ++i)
                    for (uint64_t j = 0; j < dim; ++j)
                        for (int a = 0; a < 2; ++a)
                            for (int b = 0; b < 2; ++b)
                                T[(i * 2 + a) * nd + (j * 2 + b)] = M[i * dim + j] * s[a][b];
                memcpy(M, T, sizeof(cdbl) * nd * nd);
                dim = nd;
            }
            /* tr(P A) = sum_j sum_k P[j][k] A[k][j] */
            nsum acc;
            nsum_init(&acc);
            for (uint64_t j = 0; j < N; ++j)
                for (uint64_t k = 0; k < N; ++k)
                    if (M[j * N + k] != 0) nsum_add(&acc, M[j * N + k] * A[k * N + j]);
            C[x * N + z] = scale * nsum_value(&acc);
        }
        free(M);
        free(T);
    }
    return rc;
}

/* ------------------------------------------------------------------ */
/* Direct sparse trace, Sec. II.A: P has one nonzero per row j, at     */
/* column j XOR x, with value i^{|x&z|} (-1)^{|z & (j XOR x)|}.          */
/* Loop order: mask x outer, then z, then j.                           */
/* xs == NULL: all masks, output row x.  Otherwise output row i holds   */
/* mask xs[i].                                                          */
/* ------------------------------------------------------------------ */
int oracle_direct(int n, const cdbl *A, const uint64_t *xs, uint64_t nx, cdbl *C, int nthreads)
{
    if (n < 1 || n > 16) return 1;
    const uint64_t N = 1ull << n;
    const double scale = ldexp(1.0, -n);
    if (!xs) nx = N;
    for (uint64_t i = 0; i < nx; ++i)
        if (xs && xs[i] >= N) return 1;
    set_threads(nthreads);
    int rc = 0;
#pragma omp parallel
    {
        cdbl *dx = malloc(sizeof(cdbl) * N);
        if (!dx) {
#pragma omp atomic write
            rc = 2;
        }
#pragma omp for schedule(dynamic, 1)
        for (uint64_t i = 0; i < nx; ++i) {
            if (!dx) continue;
            const uint64_t x = xs ? xs[i] : i;
            for (uint64_t j = 0; j < N; ++j) dx[j] = A[(j ^ x) * N + j]; /* A[row j^x][col j] */
            for (uint64_t z = 0; z < N; ++z) {
                nsum acc;
                nsum_init(&acc);
                for (uint64_t j = 0; j < N; ++j) {
                    /* P[j][j^x] * A[j^x][j] */
                    if (popc(z & (j ^ x)) & 1)
                        nsum_add(&acc, -dx[j]);
                    else
                        nsum_add(&acc, dx[j]);
                }
                C[i * N + z] = scale * ipow(popc(x & z)) * nsum_value(&acc);
            }
        }
        free(dx);
    }
    return rc;
}

/* ------------------------------------------------------------------ */
/* Pauli Tree Decomposition Routine, Algorithms 1-4 (Sec. III.A).      */
/*                                                                      */
/* The tree carries two arrays of length 2^n: k (column of the nonzero  */
/* in row j) and m (its value in the real-valued operator P~, where Y   */
/* is replaced by iY, Sec. II.B).  Readings of the paper taken here:    */
/*  - k holds signed offsets (column - x), so k[0] = 0 and the mask x   */
/*    accumulated along the path is added back at the leaf; this is    */
/*    the paper's k[0] = d(sigma_{n-1})...d(sigma_0) initialisation.   */
/*  - the root's children set qubit l = 0 (least significant), the     */
/*    leaves set qubit n-1 (l = tree depth - node depth - 1 in Alg. 3). */
/*  - compute_coeff is scaled by 2^-n as in the definition of Sec. II.A.*/
/* ------------------------------------------------------------------ */
typedef struct {
    int n;
    uint64_t N;
    const cdbl *A;
    cdbl *C;
    int64_t *k;
    int8_t *m;
    double scale;
} ptree;

/* Algorithm 3: the update applied when the walk enters a node with    */
/* label lab at level l.  Siblings are visited in the order I, X, Y, Z, */
/* and each rule starts from the state its left sibling left behind.   */
static void update_tree(ptree *t, int lab, int l)
{
    const uint64_t lo = 1ull << l, hi = 2ull << l;
    switch (lab) {
    case LAB_I: /* copy the top half down, shifted 2^l to the right */
        for (uint64_t j = lo; j < hi; ++j) {
            t->k[j] = t->k[j - lo] + (int64_t)lo;
            t->m[j] = t->m[j - lo];
        }
        break;
    case LAB_X: /* same values, positions shifted by -2^{l+1} */
        for (uint64_t j = lo; j < hi; ++j) t->k[j] -= (int64_t)hi;
        break;
    case LAB_Y: /* same positions, values negated (iY against X) */
        for (uint64_t j = lo; j < hi; ++j) t->m[j] = (int8_t)-t->m[j];
        break;
    default: /* Z: same values as iY, positions shifted by +2^{l+1} */
        for (uint64_t j = lo; j < hi; ++j) t->k[j] += (int64_t)hi;
        break;
    }
}

/* Algorithm 2: coeff = sum_j (-i)^{n_Y} m[j] A[k[j]][j], times 2^-n. */
static void compute_coeff(ptree *t, uint64_t x, uint64_t z, int ny)
{
    const uint64_t N = t->N;
    nsum acc;
    nsum_init(&acc);
    for (uint64_t j = 0; j < N; ++j) {
        const uint64_t row = (uint64_t)((int64_t)x + t->k[j]);
        cdbl a = t->A[row * N + j];
        nsum_add(&acc, t->m[j] > 0 ? a : -a);
    }
    t->C[x * N + z] = t->scale * ipow(3 * (ny & 3)) * nsum_value(&acc); /* (-i)^ny = i^{3 ny} */
}

/* Algorithm 4: in-order walk.  (x, z, ny) are the masks and Y count of  */
/* the labels on the path from the root to this node inclusive.         */
static void explore_node(ptree *t, int lab, int l, uint64_t x, uint64_t z, int ny)
{
    update_tree(t, lab, l);
    x |= (uint64_t)lab_d(lab) << l;
    z |= (uint64_t)lab_z(lab) << l;
    ny += (lab == LAB_Y);
    if (l == t->n - 1) {
        compute_coeff(t, x, z, ny);
        return;
    }
    for (int c = LAB_I; c <= LAB_Z; ++c) explore_node(t, c, l + 1, x, z, ny);
}

/*
 * Algorithm 1 with the forest of Sec. V.B: the tree is cut below level
 * L = min(cut, n); each of the 4^L subtrees is walked independently with
 * its own k, m arrays (one subtree per thread at a time).  Subtrees are
 * numbered by their label path written base 4 (digit l = label of qubit l);
 * only subtrees in [t0, t1) are walked, so a caller can time a bounded
 * sample.  Coefficients outside the walked subtrees are left untouched.
 */
int oracle_tree(int n, const cdbl *A, cdbl *C, int cut, uint64_t t0, uint64_t t1, int nthreads)
{
    if (n < 1 || n > 16) return 1;
    const int L = cut < n ? (cut < 0 ? 0 : cut) : n;
    const uint64_t ntrees = 1ull << (2 * L);
    if (t1 > ntrees) t1 = ntrees;
    if (t0 > t1) return 1;
    const uint64_t N = 1ull << n;
    set_threads(nthreads);
    int rc = 0;
#pragma omp parallel
    {
        ptree t;
        t.n = n;
        t.N = N;
        t.A = A;
        t.C = C;
        t.scale = ldexp(1.0, -n);
        t.k = malloc(sizeof(int64_t) * N);
        t.m = malloc(sizeof(int8_t) * N);
        if (!t.k || !t.m) {
#pragma omp atomic write
            rc = 2;
        }
#pragma omp for schedule(dynamic, 1)
        for (uint64_t tree = t0; tree < t1; ++tree) {
            if (!t.k || !t.m) continue;
            /* root state: k[0] = 0 (offset from x), m[0] = 1 */
            t.k[0] = 0;
            t.m[0] = 1;
            uint64_t x = 0, z = 0;
            int ny = 0;
            int lab = LAB_I;
            for (int l = 0; l < L; ++l) {
                lab = (int)((tree >> (2 * l)) & 3);
                /* replay the sibling chain I -> ... -> lab at this level */
                for (int s = LAB_I; s <= lab; ++s) update_tree(&t, s, l);
                x |= (uint64_t)lab_d(lab) << l;
                z |= (uint64_t)lab_z(lab) << l;
                ny += (lab == LAB_Y);
            }
            if (L == n) {
                compute_coeff(&t, x, z, ny);
            } else {
                for (int c = LAB_I; c <= LAB_Z; ++c) explore_node(&t, c, L, x, z, ny);
            }
        }
        free(t.k);
        free(t.m);
    }
    return rc;
}

/* ------------------------------------------------------------------ */
/* Inverse map A = sum_P c_P P (Sec. II.A).  Entry (r, c) of P_{x,z} is  */
/* nonzero only for x = r XOR c, with value i^{|x&z|} (-1)^{|z & c|}.    */
/* A[r][c] = scale * sum_z C[(r^c) 2^n + z] * that value.  O(8^n).       */
/* ------------------------------------------------------------------ */
int oracle_compose(int n, const cdbl *C, double scale, cdbl *A, int nthreads)
{
    if (n < 1 || n > 12) return 1;
    const uint64_t N = 1ull << n;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
    for (uint64_t r = 0; r < N; ++r) {
        for (uint64_t c = 0; c < N; ++c) {
            const uint64_t x = r ^ c;
            nsum acc;
            nsum_init(&acc);
            for (uint64_t z = 0; z < N; ++z) {
                cdbl v = ipow(popc(x & z)) * C[x * N + z];
                nsum_add(&acc, (popc(z & c) & 1) ? -v : v);
            }
            A[r * N + c] = scale * nsum_value(&acc);
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Auxiliary full check: per mask x, d_x[k] = A[k^x][k]; textbook       */
/* in-place fast Walsh-Hadamard transform over k; then                  */
/* c_{x,z} = 2^-n (-i)^{|x&z|} WHT(d_x)[z].  (Derivation: substitute     */
/* k = j in the sparse trace and pull (-1)^{|z&x|} out of the sign.)     */
/* ------------------------------------------------------------------ */
static void fwht_inplace(cdbl *v, uint64_t N)
{
    for (uint64_t h = 1; h < N; h <<= 1)
        for (uint64_t i = 0; i < N; i += 2 * h)
            for (uint64_t j = i; j < i + h; ++j) {
                cdbl a = v[j], b = v[j + h];
                v[j] = a + b;
                v[j + h] = a - b;
            }
}

int oracle_fwht(int n, const cdbl *A, const uint64_t *xs, uint64_t nx, cdbl *C, int nthreads)
{
    if (n < 1 || n > 16) return 1;
    const uint64_t N = 1ull << n;
    const double scale = ldexp(1.0, -n);
    if (!xs) nx = N;
    for (uint64_t i = 0; i < nx; ++i)
        if (xs && xs[i] >= N) return 1;
    set_threads(nthreads);
    int rc = 0;
#pragma omp parallel
    {
        cdbl *d = malloc(sizeof(cdbl) * N);
        if (!d) {
#pragma omp atomic write
            rc = 2;
        }
#pragma omp for schedule(dynamic, 1)
        for (uint64_t i = 0; i < nx; ++i) {
            if (!d) continue;
            const uint64_t x = xs ? xs[i] : i;
            for (uint64_t k = 0; k < N; ++k) d[k] = A[(k ^ x) * N + k];
            fwht_inplace(d, N);
            for (uint64_t z = 0; z < N; ++z) C[i * N + z] = scale * ipow(3 * popc(x & z)) * d[z];
        }
        free(d);
    }
    return rc;
}

/*
 * oracle_compose_fwht: the inverse map A = scale * sum_P c_P P (Sec. II.A)
 * for sizes where the direct O(8^n) sum is too slow.  Writing out the one
 * nonzero of P_{x,z} per row (value i^{|x&z|} (-1)^{|z & (j XOR x)|} at
 * column j XOR x) gives, with k = j XOR x,
 *     A[k XOR x][k] = scale * sum_z (-1)^{|z & k|} i^{|x&z|} C[x][z],
 * a textbook Walsh-Hadamard transform over z per mask x.
 *   xs == NULL: C is the whole 2^n x 2^n array and out receives all of A.
 *   otherwise:  C holds nx rows (row i = the coefficients of mask xs[i]) and
 *               out row i receives the XOR-diagonal out[i][k] = A[k XOR xs[i]][k]
 *               (so large matrices can be checked a few masks at a time).
 * Validated against oracle_compose for n <= 10 by the oracle tests.
 */
int oracle_compose_fwht(int n, const cdbl *C, const uint64_t *xs, uint64_t nx, double scale, cdbl *out,
                        int nthreads)
{
    if (n < 1 || n > 16) return 1;
    const uint64_t N = 1ull << n;
    if (!xs) nx = N;
    for (uint64_t i = 0; i < nx; ++i)
        if (xs && xs[i] >= N) return 1;
    set_threads(nthreads);
    int rc = 0;
#pragma omp parallel
    {
        cdbl *e = malloc(sizeof(cdbl) * N);
        if (!e) {
#pragma omp atomic write
            rc = 2;
        }
#pragma omp for schedule(dynamic, 1)
        for (uint64_t i = 0; i < nx; ++i) {
            if (!e) continue;
            const uint64_t x = xs ? xs[i] : i;
            for (uint64_t z = 0; z < N; ++z) e[z] = ipow(popc(x & z)) * C[i * N + z];
            fwht_inplace(e, N);
            for (uint64_t k = 0; k < N; ++k) {
                if (xs)
                    out[i * N + k] = scale * e[k];
                else
                    out[(k ^ x) * N + k] = scale * e[k];
            }
        }
        free(e);
    }
    return rc;
}

/* ------------------------------------------------------------------ */
/* Band storage (Sec. IV.A): bands[(d + s) 2^n + c] = A[c + d][c] for    */
/* d in [-s, s]; entries outside the matrix are ignored.                */
/* ------------------------------------------------------------------ */
static cdbl band_entry(const cdbl *bands, uint64_t N, int s, uint64_t r, uint64_t c)
{
    int64_t d = (int64_t)r - (int64_t)c;
    if (d < -s || d > s) return 0.0;
    return bands[(uint64_t)(d + s) * N + c];
}

/* Direct sparse trace over band storage, for the masks in xs; output   */
/* row i holds mask xs[i].                                              */
int oracle_band_direct(int n, int s, const cdbl *bands, const uint64_t *xs, uint64_t nx, cdbl *C,
                       int nthreads)
{
    if (n < 1 || n > 16 || s < 0) return 1;
    const uint64_t N = 1ull << n;
    const double scale = ldexp(1.0, -n);
    for (uint64_t i = 0; i < nx; ++i)
        if (xs[i] >= N) return 1;
    set_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (uint64_t i = 0; i < nx; ++i) {
        for (uint64_t z = 0; z < N; ++z) {
            const uint64_t x = xs[i];
            nsum acc;
            nsum_init(&acc);
            for (uint64_t j = 0; j < N; ++j) {
                cdbl a = band_entry(bands, N, s, j ^ x, j);
                if (a == 0) continue;
                nsum_add(&acc, (popc(z & (j ^ x)) & 1) ? -a : a);
            }
            C[i * N + z] = scale * ipow(popc(x & z)) * nsum_value(&acc);
        }
    }
    return 0;
}

/* Dense-gather FWHT over band storage (auxiliary full check, large n). */
int oracle_band_fwht(int n, int s, const cdbl *bands, const uint64_t *xs, uint64_t nx, cdbl *C,
                     int nthreads)
{
    if (n < 1 || n > 30 || s < 0) return 1;
    const uint64_t N = 1ull << n;
    const double scale = ldexp(1.0, -n);
    for (uint64_t i = 0; i < nx; ++i)
        if (xs[i] >= N) return 1;
    set_threads(nthreads);
    cdbl *d = malloc(sizeof(cdbl) * N);
    if (!d) return 2;
    for (uint64_t i = 0; i < nx; ++i) {
        const uint64_t x = xs[i];
#pragma omp parallel for schedule(static)
        for (uint64_t k = 0; k < N; ++k) d[k] = band_entry(bands, N, s, k ^ x, k);
        /* same textbook transform as above, with the stages' inner loops  */
        /* spread over threads                                              */
        for (uint64_t h = 1; h < N; h <<= 1) {
#pragma omp parallel for schedule(static)
            for (uint64_t p = 0; p < N / 2; ++p) {
                uint64_t j = (p / h) * 2 * h + (p % h);
                cdbl a = d[j], b = d[j + h];
                d[j] = a + b;
                d[j + h] = a - b;
            }
        }
#pragma omp parallel for schedule(static)
        for (uint64_t z = 0; z < N; ++z) C[i * N + z] = scale * ipow(3 * popc(x & z)) * d[z];
    }
    free(d);
    return 0;
}

/* Brute-force mask enumeration: x is reachable by a band of half-width */
/* s iff some in-band entry (r, c) has r XOR c = x.  Writes the sorted  */
/* masks to out (capacity cap) and their number to *count.               */
int oracle_band_masks(int n, int s, uint64_t *out, uint64_t cap, uint64_t *count)
{
    if (n < 1 || n > 30 || s < 0) return 1;
    const uint64_t N = 1ull << n;
    unsigned char *hit = calloc(N, 1);
    if (!hit) return 2;
    for (uint64_t r = 0; r < N; ++r)
        for (int64_t d = -s; d <= s; ++d) {
            int64_t c = (int64_t)r - d;
            if (c < 0 || c >= (int64_t)N) continue;
            hit[r ^ (uint64_t)c] = 1;
        }
    uint64_t cnt = 0;
    for (uint64_t x = 0; x < N; ++x)
        if (hit[x]) {
            if (cnt < cap && out) out[cnt] = x;
            ++cnt;
        }
    free(hit);
    *count = cnt;
    return cnt > cap ? 3 : 0;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
