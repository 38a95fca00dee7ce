/*
 * rchol_oracle.c -- sequential FP64 reference for randomized approximate
 * Cholesky (rchol, as parallelised by ParAC, arXiv 2505.02977) and for PCG
 * preconditioned by the resulting factor.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness oracle: it is
 * compiled, loaded and called only by the test-suite, by the package's
 * smoke check and by the benchmark's CPU-baseline leg.  The library's
 * product path never links, loads or calls it, and it shares no source,
 * header, table or helper with the CUDA implementation.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fPIC -shared
 * (-ffp-contract=off matters: aarch64 GCC would otherwise fuse a*b+c).
 *
 * What it computes, step by step (paper references are to the ParAC paper):
 *   ingest      Sec. V "Experimental Methodology": Laplacian/SDDM sign
 *               convention; SDDM rows with positive excess get an edge to an
 *               appended ground node.  Ordering (Sec. V "Ordering") relabels
 *               vertices; only the strict lower triangle (row label > column
 *               label) is kept, as edge weights w = -l_ij > 0.
 *   factor      Alg. 1 outer loop with Alg. 2 (SampleClique) per pivot, in
 *               the scaled form L ~ F D F^T of Sec. IV (G = F D^{1/2}),
 *               using the suffix-sum formulation of Alg. 3.  Pivots are taken
 *               in label order, which is a valid order of the dependency DAG
 *               of Sec. III (every fill edge joins two labels above the pivot).
 *   tracked     The same eliminations scheduled by the dependency counters of
 *               Sec. III ("Proposed Tracking Strategy"): d(i) counts lower
 *               incident edges with multiplicity, sampled-edge increments are
 *               applied before the pivot-edge decrements, and a vertex enters
 *               the ready set on a positive-to-zero transition.  Any ready
 *               vertex may be picked next (a seeded random choice); Sec. III
 *               "Distribution Preservation" says the result cannot depend on it.
 *   pcg         Standard preconditioned conjugate gradients (Sec. V) with
 *               M^{-1} = P^T F^{-T} D^+ F^{-1} P, the factor applied in FP64
 *               or, in the mixed form (readings M1-M5 below, next to the
 *               code), stored and applied in FP32 inside FP64 recurrences.
 *
 * Readings of points the paper leaves open (each is a definition here, and
 * the CUDA path must reproduce it exactly):
 *   R1 merge order.  A pivot's gathered entries are sorted by (row ascending,
 *      IEEE bit pattern of w ascending); each run of equal rows is summed left
 *      to right, and m_u is the run length (the multiplicity of Sec. III).
 *   R2 weight order.  Merged entries are sorted by (w bits ascending, row
 *      ascending) -- Alg. 2 says "ascending |l_ki|" with no tie rule.
 *   R3 suffix sums.  S[i] = sum_{q >= i} w_q (0-based), formed only by the
 *      pairings of a 32-wide Hillis-Steele inclusive scan over the reversed
 *      array a[t] = w[d-1-t], tile by tile (tail tile padded with +0.0), each
 *      tile's lanes then adding the carry of the previous tiles (carry_0 =
 *      +0.0, carry_{j+1} = last lane of tile j after its carry add).
 *      D_k = S[0] (Alg. 3: D(k,k) = sum of the neighbour weights).
 *   R4 sampling.  For slot p = 1..d-1 (1-based, as in Alg. 3), Philox4x64-10
 *      with counter (k, p, sys, 0) and key (seed, 0) gives o0; the uniform is
 *      v = ((o0 >> 11) + 1) * 2^-53 in (0, 1]; R = S[p] * v (0-based S[p] is
 *      the 1-based S[p+1]); the sampled neighbour is the LARGEST 0-based index
 *      j in [p, d-1] with S[j] >= R.  In exact arithmetic this picks j with
 *      probability w_j / S[p], the rule of Alg. 2/3.
 *   R5 fill weight.  c = (S[p] * w_{p-1}) / D_k, multiply then divide
 *      (Alg. 3: S[p+1] |l_ku| / l_kk), appended as (row = max(u,v), c) to the
 *      column of min(u,v).
 *   R6 factor column.  F(u,k) = -w_u / D_k (one IEEE division), rows ascending;
 *      N_k empty gives D_k = 0 and an empty column (Alg. 3).
 *   R7 SDDM excess.  e_j = sequential sum of the stored entries of column j in
 *      stored order, diagonal included.  e_j > 1e-12 * l_jj adds a ground edge
 *      of weight e_j; e_j < -1e-12 * l_jj is not diagonally dominant.
 *   R8 dependency counters start at the number of stored lower entries of each
 *      row (with multiplicity; equals Sec. III's d_0 for duplicate-free input).
 *   R9 AC(k) (Sec. VI: two samples per original entry, after Gao, Kyng and
 *      Spielman).  Each strict-lower entry of the ingested matrix, ground
 *      edges included, is split into k parallel entries of weight RN(w / k);
 *      the elimination then runs on the multigraph: every gathered entry is
 *      a clique-tree slot of its own (R2-R5 over the g entries instead of the
 *      d merged ones; D_k = S[0] of that scan), a sample pairing two entries
 *      of one row is a self-loop and adds nothing, and the factor column and
 *      the counters use the merged rows of R1.  Unlike MS(k) (orc_eliminate_k),
 *      fill entries are not resampled k times: each slot draws once.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOT_SDD = 2, ORC_ENOMEM = 3 };
enum { ORC_KIND_AUTO = 0, ORC_KIND_LAPLACIAN = 1, ORC_KIND_SDDM = 2 };

#define ORC_SDDM_TOL 1e-12

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11).  Multipliers and Weyl key increments are the    */
/* ones that paper specifies for the 4x64 variant.                           */
/* ------------------------------------------------------------------------ */
void orc_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4])
{
    uint64_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B97F4A7C15ULL;
            k1 += 0xBB67AE8584CAA73BULL;
        }
        unsigned __int128 p0 = (unsigned __int128)0xD2E7470EE14C6C93ULL * x0;
        unsigned __int128 p1 = (unsigned __int128)0xCA5A826395121157ULL * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t n0 = hi1 ^ x1 ^ k0;
        uint64_t n2 = hi0 ^ x3 ^ k1;
        x0 = n0; x1 = lo1; x2 = n2; x3 = lo0;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* R4: the uniform in (0,1] drawn for sample q of slot p of pivot k of
 * system sys (q = 0 for the plain method; MS(k) draws q = 0..k-1). */
double orc_slot_uniform_s(uint64_t seed, uint64_t k, uint64_t p, uint64_t sys, uint64_t q)
{
    uint64_t ctr[4] = { k, p, sys, q }, key[2] = { seed, 0 }, o[4];
    orc_philox4x64_10(ctr, key, o);
    uint64_t m53 = o[0] >> 11;
    return (double)(m53 + 1) * 0x1.0p-53;
}

double orc_slot_uniform(uint64_t seed, uint64_t k, uint64_t p, uint64_t sys)
{
    return orc_slot_uniform_s(seed, k, p, sys, 0);
}

/* ------------------------------------------------------------------------ */
/* Canonical suffix sums (R3).                                               */
/* ------------------------------------------------------------------------ */
void orc_suffix_scan(int64_t d, const double *w, double *S)
{
    double carry = 0.0;
    for (int64_t base = 0; base < d; base += 32) {
        double x[32], prev[32];
        for (int i = 0; i < 32; ++i) {
            int64_t t = base + i;
            x[i] = (t < d) ? w[d - 1 - t] : 0.0;
        }
        for (int off = 1; off < 32; off <<= 1) {
            memcpy(prev, x, sizeof x);
            for (int i = off; i < 32; ++i) x[i] = prev[i] + prev[i - off];
        }
        for (int i = 0; i < 32; ++i) x[i] = x[i] + carry;
        carry = x[31];
        for (int i = 0; i < 32; ++i) {
            int64_t t = base + i;
            if (t < d) S[d - 1 - t] = x[i];
        }
    }
}

/* R4 search, literal form: the largest j in [lo, d-1] with S[j] >= R. */
int64_t orc_pick_bruteforce(int64_t d, const double *S, int64_t lo, double R)
{
    for (int64_t j = d - 1; j >= lo; --j)
        if (S[j] >= R) return j;
    return -1;
}

/* R4 search as used by the factor.  M[j] = max_{q >= j} S[q] is exact (no
 * rounding), non-increasing, and M[j] >= R holds iff some q >= j has
 * S[q] >= R; so the largest j with M[j] >= R is the largest j with
 * S[j] >= R.  A binary search on M finds it in O(log d). */
int64_t orc_pick_search(int64_t d, const double *M, int64_t lo, double R)
{
    if (lo > d - 1 || !(M[lo] >= R)) return -1;
    int64_t a = lo, b = d - 1;          /* invariant: M[a] >= R */
    while (a < b) {
        int64_t mid = a + (b - a + 1) / 2;
        if (M[mid] >= R) a = mid; else b = mid - 1;
    }
    return a;
}

/* ------------------------------------------------------------------------ */
/* One pivot: gather -> merge -> D, F column -> weight sort -> scan ->       */
/* sample (Alg. 2 / Alg. 3 body).                                            */
/* ------------------------------------------------------------------------ */
typedef struct { int32_t row; uint64_t bits; double w; } orc_ent;

static uint64_t dbits(double x) { uint64_t b; memcpy(&b, &x, 8); return b; }

static int cmp_row_bits(const void *pa, const void *pb)
{
    const orc_ent *a = pa, *b = pb;
    if (a->row != b->row) return a->row < b->row ? -1 : 1;
    if (a->bits != b->bits) return a->bits < b->bits ? -1 : 1;
    return 0;
}

static int cmp_bits_row(const void *pa, const void *pb)
{
    const orc_ent *a = pa, *b = pb;
    if (a->bits != b->bits) return a->bits < b->bits ? -1 : 1;
    if (a->row != b->row) return a->row < b->row ? -1 : 1;
    return 0;
}

/* Results of eliminating one pivot.  Arrays are caller-provided with room
 * for g entries (g = number of gathered entries). */
typedef struct {
    int64_t d;          /* merged neighbour count */
    double D;           /* pivot */
    int32_t *mrow;      /* merged rows, ascending            [g] */
    double  *mw;        /* merged weights                    [g] */
    int32_t *mmult;     /* multiplicities                    [g] */
    double  *fval;      /* F(u,k) for mrow order             [g] */
    int32_t *slo, *shi; /* sampled edges (min, max label)    [ksamp * g], sample q of slot p at q*(d-1) + p-1 */
    double  *sc;        /* sampled edge weights              [ksamp * g] */
    int64_t *spick;     /* 0-based weight-order index picked [ksamp * g] */
    int64_t ns;         /* sampled slots written (entries with slo < 0 are self-loops, no edge) */
} orc_step;

/* Eliminate pivot k whose gathered entries are (rows[i], w[i]), i < g.
 * ksamp samples per slot: per-slot multi-sampling MS(ksamp), where every slot
 * of the clique tree, at every pivot, draws ksamp independent neighbours with
 * counters (k, p, sys, q), q < ksamp, each edge weighted c_p / ksamp; ksamp =
 * 1 is Alg. 2.  This is NOT Sec. VI's AC(2) (after Gao-Kyng-Spielman), which
 * doubles the samples of the input matrix's own entries only:
 * MS(k) also multiplies the samples of fill-derived entries, so its fill
 * compounds from pivot to pivot. */
static int orc_eliminate_k(int64_t g, const int32_t *rows, const double *w, uint64_t seed,
                           uint64_t k, uint64_t sys, int ksamp, orc_step *st)
{
    orc_ent *e = malloc(sizeof(orc_ent) * (size_t)(g > 0 ? g : 1));
    orc_ent *s = malloc(sizeof(orc_ent) * (size_t)(g > 0 ? g : 1));
    double *S = malloc(sizeof(double) * (size_t)(g > 0 ? g : 1));
    double *M = malloc(sizeof(double) * (size_t)(g > 0 ? g : 1));
    if (!e || !s || !S || !M) { free(e); free(s); free(S); free(M); return ORC_ENOMEM; }

    for (int64_t i = 0; i < g; ++i) { e[i].row = rows[i]; e[i].w = w[i]; e[i].bits = dbits(w[i]); }
    qsort(e, (size_t)g, sizeof(orc_ent), cmp_row_bits);            /* R1 */

    int64_t d = 0;
    for (int64_t i = 0; i < g;) {
        int64_t j = i;
        double sum = e[i].w;
        while (j + 1 < g && e[j + 1].row == e[i].row) { ++j; sum = sum + e[j].w; }
        st->mrow[d] = e[i].row; st->mw[d] = sum; st->mmult[d] = (int32_t)(j - i + 1);
        ++d;
        i = j + 1;
    }
    st->d = d;
    st->ns = (int64_t)ksamp * (d > 0 ? d - 1 : 0);
    if (d == 0) { st->D = 0.0; free(e); free(s); free(S); free(M); return ORC_OK; }

    for (int64_t i = 0; i < d; ++i) { s[i].row = st->mrow[i]; s[i].w = st->mw[i]; s[i].bits = dbits(st->mw[i]); }
    qsort(s, (size_t)d, sizeof(orc_ent), cmp_bits_row);            /* R2 */

    double *ws = malloc(sizeof(double) * (size_t)d);
    if (!ws) { free(e); free(s); free(S); free(M); return ORC_ENOMEM; }
    for (int64_t i = 0; i < d; ++i) ws[i] = s[i].w;
    orc_suffix_scan(d, ws, S);                                     /* R3 */
    free(ws);
    double D = S[0];
    st->D = D;
    for (int64_t i = 0; i < d; ++i) st->fval[i] = -st->mw[i] / D;  /* R6 */

    M[d - 1] = S[d - 1];
    for (int64_t j = d - 2; j >= 0; --j) M[j] = S[j] > M[j + 1] ? S[j] : M[j + 1];

    for (int q = 0; q < ksamp; ++q) {
        for (int64_t p = 1; p <= d - 1; ++p) {                     /* R4, R5 */
            double v = orc_slot_uniform_s(seed, k, (uint64_t)p, sys, (uint64_t)q);
            double R = S[p] * v;
            int64_t j = orc_pick_search(d, M, p, R);
            int32_t u = s[p - 1].row, x = s[j].row;
            double c = (S[p] * s[p - 1].w) / D;
            if (ksamp > 1) c = c / (double)ksamp;
            int64_t at = (int64_t)q * (d - 1) + (p - 1);
            st->slo[at] = u < x ? u : x;
            st->shi[at] = u < x ? x : u;
            st->sc[at] = c;
            st->spick[at] = j;
        }
    }
    free(e); free(s); free(S); free(M);
    return ORC_OK;
}

/* AC(k) of Sec. VI (after Gao, Kyng and Spielman): the input's own entries
 * are split into k parallel entries of weight w/k before the elimination
 * (orc_factor_run_ac), and the elimination runs on the multigraph.  At a
 * pivot every gathered entry -- an original copy or a fill entry -- is its
 * own clique-tree slot: the entries are sorted by (weight bits, row) without
 * merging (R2 over entries; equal keys are identical entries, so their
 * order does not matter), the canonical suffix scan runs over all g of them
 * (R3), D_k = S[1], and slot p = 1..g-1 samples by R4/R5 among the later
 * entries.  A sample that pairs two entries of the same row is a self-loop
 * and adds nothing (its Laplacian term is zero): no fill, no counter
 * increment.  The factor column and the counters use the merged rows (R1):
 * F(u,k) = -(run sum of u's entries) / D_k, multiplicity m_u.  slo = shi =
 * -1 marks a self-loop; sc holds every slot's weight c_p. */
static int orc_eliminate_ac(int64_t g, const int32_t *rows, const double *w, uint64_t seed,
                            uint64_t k, uint64_t sys, orc_step *st)
{
    orc_ent *e = malloc(sizeof(orc_ent) * (size_t)(g > 0 ? g : 1));
    double *S = malloc(sizeof(double) * (size_t)(g > 0 ? g : 1));
    double *M = malloc(sizeof(double) * (size_t)(g > 0 ? g : 1));
    double *ws = malloc(sizeof(double) * (size_t)(g > 0 ? g : 1));
    if (!e || !S || !M || !ws) { free(e); free(S); free(M); free(ws); return ORC_ENOMEM; }

    for (int64_t i = 0; i < g; ++i) { e[i].row = rows[i]; e[i].w = w[i]; e[i].bits = dbits(w[i]); }
    qsort(e, (size_t)g, sizeof(orc_ent), cmp_row_bits);            /* R1: merged rows for F and the counters */
    int64_t d = 0;
    for (int64_t i = 0; i < g;) {
        int64_t j = i;
        double sum = e[i].w;
        while (j + 1 < g && e[j + 1].row == e[i].row) { ++j; sum = sum + e[j].w; }
        st->mrow[d] = e[i].row; st->mw[d] = sum; st->mmult[d] = (int32_t)(j - i + 1);
        ++d;
        i = j + 1;
    }
    st->d = d;
    st->ns = g > 0 ? g - 1 : 0;
    if (d == 0) { st->D = 0.0; free(e); free(S); free(M); free(ws); return ORC_OK; }

    qsort(e, (size_t)g, sizeof(orc_ent), cmp_bits_row);            /* R2 over the entries */
    for (int64_t i = 0; i < g; ++i) ws[i] = e[i].w;
    orc_suffix_scan(g, ws, S);                                     /* R3 over the entries */
    const double D = S[0];
    st->D = D;
    for (int64_t i = 0; i < d; ++i) st->fval[i] = -st->mw[i] / D;

    M[g - 1] = S[g - 1];
    for (int64_t j = g - 2; j >= 0; --j) M[j] = S[j] > M[j + 1] ? S[j] : M[j + 1];
    for (int64_t p = 1; p <= g - 1; ++p) {                         /* R4, R5 per entry slot */
        double v = orc_slot_uniform_s(seed, k, (uint64_t)p, sys, 0);
        double R = S[p] * v;
        int64_t j = orc_pick_search(g, M, p, R);
        int32_t u = e[p - 1].row, x = e[j].row;
        double c = (S[p] * e[p - 1].w) / D;
        st->sc[p - 1] = c;
        st->spick[p - 1] = j;
        if (u == x) { st->slo[p - 1] = -1; st->shi[p - 1] = -1; }
        else { st->slo[p - 1] = u < x ? u : x; st->shi[p - 1] = u < x ? x : u; }
    }
    free(e); free(S); free(M); free(ws);
    return ORC_OK;
}

int orc_eliminate(int64_t g, const int32_t *rows, const double *w, uint64_t seed,
                  uint64_t k, uint64_t sys, orc_step *st)
{
    return orc_eliminate_k(g, rows, w, seed, k, sys, 1, st);
}

/* ------------------------------------------------------------------------ */
/* Ingest (a1): validation, ordering, strict lower part, ground node.       */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n;          /* labels, ground included */
    int64_t n_orig;
    int has_ground;
    int64_t *colptr;
    int32_t *row;
    double *w;
} orc_low;

static void low_free(orc_low *L) { free(L->colptr); free(L->row); free(L->w); memset(L, 0, sizeof *L); }

int orc_ingest(int64_t n, const int64_t *colptr, const int32_t *rowind, const double *val,
               const int32_t *ordering, int kind, orc_low *out)
{
    memset(out, 0, sizeof *out);
    if (n < 0 || n > 0x7ffffffeLL || !colptr) return ORC_EINVAL;
    if (colptr[0] != 0) return ORC_EINVAL;
    for (int64_t j = 0; j < n; ++j) if (colptr[j + 1] < colptr[j]) return ORC_EINVAL;
    int64_t nnz = colptr[n];
    for (int64_t t = 0; t < nnz; ++t) if (rowind[t] < 0 || rowind[t] >= n) return ORC_EINVAL;

    int32_t *iperm = malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!iperm) return ORC_ENOMEM;
    if (ordering) {
        for (int64_t i = 0; i < n; ++i) iperm[i] = -1;
        for (int64_t k = 0; k < n; ++k) {
            int32_t v = ordering[k];
            if (v < 0 || v >= n || iperm[v] != -1) { free(iperm); return ORC_EINVAL; }
            iperm[v] = (int32_t)k;
        }
    } else {
        for (int64_t i = 0; i < n; ++i) iperm[i] = (int32_t)i;
    }

    /* R7 excess, sign checks */
    double *exc = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *dia = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!exc || !dia) { free(iperm); free(exc); free(dia); return ORC_ENOMEM; }
    int any_excess = 0;
    for (int64_t j = 0; j < n; ++j) {
        double e = 0.0, dg = 0.0;
        for (int64_t t = colptr[j]; t < colptr[j + 1]; ++t) {
            double v = val[t];
            if (rowind[t] == j) dg = dg + v;
            else if (v > 0.0) { free(iperm); free(exc); free(dia); return ORC_ENOT_SDD; }
            e = e + v;
        }
        exc[j] = e; dia[j] = dg;
        if (e < -ORC_SDDM_TOL * dg || (e < 0.0 && dg <= 0.0)) { free(iperm); free(exc); free(dia); return ORC_ENOT_SDD; }
        if (e > ORC_SDDM_TOL * dg) any_excess = 1;
    }
    int ground;
    if (kind == ORC_KIND_SDDM) ground = 1;
    else if (kind == ORC_KIND_LAPLACIAN) {
        if (any_excess) { free(iperm); free(exc); free(dia); return ORC_EINVAL; }
        ground = 0;
    } else if (kind == ORC_KIND_AUTO) ground = any_excess;
    else { free(iperm); free(exc); free(dia); return ORC_EINVAL; }

    int64_t nl = n + (ground ? 1 : 0);
    int64_t *cnt = calloc((size_t)nl + 1, sizeof(int64_t));
    if (!cnt) { free(iperm); free(exc); free(dia); return ORC_ENOMEM; }
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t t = colptr[j]; t < colptr[j + 1]; ++t) {
            int32_t i = rowind[t];
            if (i == j || val[t] == 0.0) continue;
            if (iperm[i] > iperm[j]) cnt[iperm[j]]++;
        }
        if (ground && exc[j] > ORC_SDDM_TOL * dia[j]) cnt[iperm[j]]++;
    }
    int64_t *cp = malloc(sizeof(int64_t) * (size_t)(nl + 1));
    if (!cp) { free(iperm); free(exc); free(dia); free(cnt); return ORC_ENOMEM; }
    cp[0] = 0;
    for (int64_t c = 0; c < nl; ++c) cp[c + 1] = cp[c] + cnt[c];
    int64_t m = cp[nl];
    int32_t *row = malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    double *w = malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    if (!row || !w) { free(iperm); free(exc); free(dia); free(cnt); free(cp); free(row); free(w); return ORC_ENOMEM; }
    for (int64_t c = 0; c < nl; ++c) cnt[c] = cp[c];
    for (int64_t j = 0; j < n; ++j) {
        int32_t lj = iperm[j];
        for (int64_t t = colptr[j]; t < colptr[j + 1]; ++t) {
            int32_t i = rowind[t];
            if (i == j || val[t] == 0.0) continue;
            if (iperm[i] > lj) { row[cnt[lj]] = iperm[i]; w[cnt[lj]] = -val[t]; cnt[lj]++; }
        }
        if (ground && exc[j] > ORC_SDDM_TOL * dia[j]) { row[cnt[lj]] = (int32_t)n; w[cnt[lj]] = exc[j]; cnt[lj]++; }
    }
    free(iperm); free(exc); free(dia); free(cnt);
    out->n = nl; out->n_orig = n; out->has_ground = ground;
    out->colptr = cp; out->row = row; out->w = w;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Factor (Alg. 1 over labels).                                              */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n;              /* output labels (ground removed) */
    int has_ground;
    int64_t *colptr;        /* CSC of strict-lower unit F, rows ascending */
    int32_t *row;
    double *val;
    double *D;              /* n */
    int64_t nnz_low_in;     /* strict-lower input entries incl. ground edges */
    int64_t fill;           /* sampled edges appended */
    int64_t nnz_all;        /* sum of d_k over every label incl. ground */
    int64_t max_gather;     /* largest gathered list */
    int64_t depth;          /* critical path of the realised dependency DAG */
    int64_t violations;     /* tracked mode: invariant violations observed */
} orc_factor;

typedef struct { int64_t cnt, cap; int32_t *row; double *w; } orc_fillcol;

static int fill_push(orc_fillcol *c, int32_t r, double w)
{
    if (c->cnt == c->cap) {
        int64_t nc = c->cap ? 2 * c->cap : 8;
        int32_t *nr = realloc(c->row, sizeof(int32_t) * (size_t)nc);
        if (!nr) return ORC_ENOMEM;
        c->row = nr;
        double *nw = realloc(c->w, sizeof(double) * (size_t)nc);
        if (!nw) return ORC_ENOMEM;
        c->w = nw;
        c->cap = nc;
    }
    c->row[c->cnt] = r; c->w[c->cnt] = w; c->cnt++;
    return ORC_OK;
}

typedef struct {
    orc_low L;
    orc_fillcol *fill;
    int64_t *fcount;        /* d_k per label */
    int32_t **frow; double **fval;
    double *D;
    int64_t *level;         /* dependency-DAG level per label */
    int64_t max_gather, nfill, nnz_all;
    int ksamp;              /* samples per clique-tree slot (MS(ksamp)); 1 = Alg. 2 */
    int ac;                 /* nonzero: AC(k) multigraph elimination (orc_eliminate_ac) */
} orc_state;

static void state_free(orc_state *S)
{
    if (S->fill) for (int64_t c = 0; c < S->L.n; ++c) { free(S->fill[c].row); free(S->fill[c].w); }
    if (S->frow) for (int64_t c = 0; c < S->L.n; ++c) { free(S->frow[c]); free(S->fval[c]); }
    free(S->fill); free(S->fcount); free(S->frow); free(S->fval); free(S->D); free(S->level);
    low_free(&S->L);
}

static int state_init(orc_state *S)
{
    int64_t nl = S->L.n;
    size_t nn = (size_t)(nl > 0 ? nl : 1);
    S->fill = calloc(nn, sizeof(orc_fillcol));
    S->fcount = calloc(nn, sizeof(int64_t));
    S->frow = calloc(nn, sizeof(int32_t *));
    S->fval = calloc(nn, sizeof(double *));
    S->D = calloc(nn, sizeof(double));
    S->level = calloc(nn, sizeof(int64_t));
    if (!S->fill || !S->fcount || !S->frow || !S->fval || !S->D || !S->level) return ORC_ENOMEM;
    return ORC_OK;
}

/* Eliminate label k in state S; on success optionally report the merged
 * rows and multiplicities and the sampled edges through st_out. */
static int state_eliminate(orc_state *S, int64_t k, uint64_t seed, uint64_t sys, orc_step *st_keep)
{
    int64_t o0 = S->L.colptr[k], o1 = S->L.colptr[k + 1];
    int64_t g = (o1 - o0) + S->fill[k].cnt;
    if (g > S->max_gather) S->max_gather = g;
    size_t gg = (size_t)(g > 0 ? g : 1);
    const int ks = S->ksamp > 0 ? S->ksamp : 1;
    size_t gs = gg * (size_t)ks;
    int32_t *rows = malloc(sizeof(int32_t) * gg);
    double *w = malloc(sizeof(double) * gg);
    orc_step st;
    st.mrow = malloc(sizeof(int32_t) * gg); st.mw = malloc(sizeof(double) * gg);
    st.mmult = malloc(sizeof(int32_t) * gg); st.fval = malloc(sizeof(double) * gg);
    st.slo = malloc(sizeof(int32_t) * gs); st.shi = malloc(sizeof(int32_t) * gs);
    st.sc = malloc(sizeof(double) * gs); st.spick = malloc(sizeof(int64_t) * gs);
    if (!rows || !w || !st.mrow || !st.mw || !st.mmult || !st.fval || !st.slo || !st.shi || !st.sc || !st.spick)
        return ORC_ENOMEM;
    int64_t t = 0;
    for (int64_t q = o0; q < o1; ++q) { rows[t] = S->L.row[q]; w[t] = S->L.w[q]; ++t; }
    for (int64_t q = 0; q < S->fill[k].cnt; ++q) { rows[t] = S->fill[k].row[q]; w[t] = S->fill[k].w[q]; ++t; }
    free(S->fill[k].row); free(S->fill[k].w); memset(&S->fill[k], 0, sizeof(orc_fillcol));

    int rc = S->ac ? orc_eliminate_ac(g, rows, w, seed, (uint64_t)k, sys, &st)
                   : orc_eliminate_k(g, rows, w, seed, (uint64_t)k, sys, ks, &st);
    free(rows); free(w);
    if (rc) return rc;
    S->D[k] = st.D;
    S->fcount[k] = st.d;
    S->nnz_all += st.d;
    S->frow[k] = malloc(sizeof(int32_t) * (size_t)(st.d > 0 ? st.d : 1));
    S->fval[k] = malloc(sizeof(double) * (size_t)(st.d > 0 ? st.d : 1));
    if (!S->frow[k] || !S->fval[k]) return ORC_ENOMEM;
    memcpy(S->frow[k], st.mrow, sizeof(int32_t) * (size_t)st.d);
    memcpy(S->fval[k], st.fval, sizeof(double) * (size_t)st.d);
    int64_t lk = S->level[k] + 1;
    for (int64_t i = 0; i < st.d; ++i)
        if (S->level[st.mrow[i]] < lk) S->level[st.mrow[i]] = lk;
    const int64_t nsamp = st.ns;
    for (int64_t p = 0; p < nsamp; ++p) {
        if (st.slo[p] < 0) continue;                      /* AC(k): a self-loop adds nothing */
        rc = fill_push(&S->fill[st.slo[p]], st.shi[p], st.sc[p]);
        if (rc) return rc;
        S->nfill++;
    }
    if (st_keep) {
        *st_keep = st;
    } else {
        free(st.mrow); free(st.mw); free(st.mmult); free(st.fval);
        free(st.slo); free(st.shi); free(st.sc); free(st.spick);
    }
    return ORC_OK;
}

static void step_free(orc_step *st)
{
    free(st->mrow); free(st->mw); free(st->mmult); free(st->fval);
    free(st->slo); free(st->shi); free(st->sc); free(st->spick);
}

static int state_to_factor(orc_state *S, orc_factor **out)
{
    orc_factor *F = calloc(1, sizeof(orc_factor));
    if (!F) return ORC_ENOMEM;
    int64_t n = S->L.n_orig;
    F->n = n; F->has_ground = S->L.has_ground;
    F->colptr = malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!F->colptr) { free(F); return ORC_ENOMEM; }
    F->colptr[0] = 0;
    for (int64_t k = 0; k < n; ++k) {
        int64_t dk = S->fcount[k];
        if (dk > 0 && S->frow[k][dk - 1] >= n) dk--;   /* drop the ground row (largest label) */
        F->colptr[k + 1] = F->colptr[k] + dk;
    }
    int64_t nnz = F->colptr[n];
    F->row = malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    F->val = malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
    F->D = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!F->row || !F->val || !F->D) return ORC_ENOMEM;
    for (int64_t k = 0; k < n; ++k) {
        int64_t c0 = F->colptr[k], len = F->colptr[k + 1] - c0;
        if (len) {
            memcpy(F->row + c0, S->frow[k], sizeof(int32_t) * (size_t)len);
            memcpy(F->val + c0, S->fval[k], sizeof(double) * (size_t)len);
        }
        F->D[k] = S->D[k];
    }
    F->nnz_low_in = S->L.colptr[S->L.n];
    F->fill = S->nfill;
    F->nnz_all = S->nnz_all;
    F->max_gather = S->max_gather;
    int64_t depth = 0;
    for (int64_t k = 0; k < S->L.n; ++k) if (S->level[k] + 1 > depth) depth = S->level[k] + 1;
    F->depth = depth;
    *out = F;
    return ORC_OK;
}

int orc_factor_run_k(int64_t n, const int64_t *colptr, const int32_t *rowind, const double *val,
                     const int32_t *ordering, int kind, uint64_t seed, uint64_t sys, int ksamp, orc_factor **out)
{
    *out = NULL;
    if (ksamp < 1) return ORC_EINVAL;
    orc_state S;
    memset(&S, 0, sizeof S);
    S.ksamp = ksamp;
    int rc = orc_ingest(n, colptr, rowind, val, ordering, kind, &S.L);
    if (rc) return rc;
    rc = state_init(&S);
    for (int64_t k = 0; !rc && k < S.L.n; ++k) rc = state_eliminate(&S, k, seed, sys, NULL);
    if (!rc) rc = state_to_factor(&S, out);
    state_free(&S);
    return rc;
}

/* Every strict-lower entry of L split into k parallel entries of weight
 * RN(w / k), in place of the entry (AC(k), reading R9). */
static int low_split(orc_low *L, int k)
{
    const int64_t nl = L->n, m = L->colptr[nl];
    int64_t *cp = malloc(sizeof(int64_t) * (size_t)(nl + 1));
    int32_t *row = malloc(sizeof(int32_t) * (size_t)(m * k > 0 ? m * k : 1));
    double *w = malloc(sizeof(double) * (size_t)(m * k > 0 ? m * k : 1));
    if (!cp || !row || !w) { free(cp); free(row); free(w); return ORC_ENOMEM; }
    cp[0] = 0;
    for (int64_t c = 0; c < nl; ++c) {
        int64_t t = cp[c];
        for (int64_t q = L->colptr[c]; q < L->colptr[c + 1]; ++q)
            for (int r = 0; r < k; ++r) { row[t] = L->row[q]; w[t] = L->w[q] / (double)k; ++t; }
        cp[c + 1] = t;
    }
    free(L->colptr); free(L->row); free(L->w);
    L->colptr = cp; L->row = row; L->w = w;
    return ORC_OK;
}

/* AC(k): every strict-lower entry of the ingested matrix (ground edges
 * included) split into k parallel entries of weight RN(w / k), then the
 * multigraph elimination of orc_eliminate_ac. */
int orc_factor_run_ac(int64_t n, const int64_t *colptr, const int32_t *rowind, const double *val,
                      const int32_t *ordering, int kind, uint64_t seed, uint64_t sys, int ksplit, orc_factor **out)
{
    *out = NULL;
    if (ksplit < 1) return ORC_EINVAL;
    orc_state S;
    memset(&S, 0, sizeof S);
    S.ksamp = 1;
    S.ac = 1;
    int rc = orc_ingest(n, colptr, rowind, val, ordering, kind, &S.L);
    if (rc) return rc;
    rc = low_split(&S.L, ksplit);
    if (rc) { low_free(&S.L); return rc; }
    rc = state_init(&S);
    for (int64_t k = 0; !rc && k < S.L.n; ++k) rc = state_eliminate(&S, k, seed, sys, NULL);
    if (!rc) rc = state_to_factor(&S, out);
    state_free(&S);
    return rc;
}

int orc_factor_run(int64_t n, const int64_t *colptr, const int32_t *rowind, const double *val,
                   const int32_t *ordering, int kind, uint64_t seed, uint64_t sys, orc_factor **out)
{
    return orc_factor_run_k(n, colptr, rowind, val, ordering, kind, seed, sys, 1, out);
}

/* ------------------------------------------------------------------------ */
/* Dependency counters (Sec. III).                                           */
/* ------------------------------------------------------------------------ */

/* One pivot's counter update, in the paper's order: for every sampled edge
 * (a,b), dp[max(a,b)] += 1 (a < 0 marks an AC(k) self-loop: no edge); then
 * for every merged neighbour u with
 * multiplicity m, r = dp[u]; dp[u] -= m; u is enqueued when r == m (a
 * positive-to-zero transition).  If deletes_first is nonzero the two phases
 * are swapped and a vertex is enqueued whenever its counter reads zero
 * after the delete phase (the hazard of Sec. III; used only by tests).
 * Returns the number of enqueued vertices written to enq. */
int64_t orc_dp_update(int32_t *dp, int64_t nsamp, const int32_t *sa, const int32_t *sb,
                      int64_t nnbr, const int32_t *nbr, const int32_t *mult, int32_t *enq,
                      int deletes_first)
{
    int64_t ne = 0;
    if (!deletes_first) {
        for (int64_t s = 0; s < nsamp; ++s) if (sa[s] >= 0) dp[sa[s] > sb[s] ? sa[s] : sb[s]] += 1;
        for (int64_t i = 0; i < nnbr; ++i) {
            int32_t r = dp[nbr[i]];
            dp[nbr[i]] = r - mult[i];
            if (r == mult[i]) enq[ne++] = nbr[i];
        }
    } else {
        for (int64_t i = 0; i < nnbr; ++i) {
            dp[nbr[i]] -= mult[i];
            if (dp[nbr[i]] == 0) enq[ne++] = nbr[i];
        }
        for (int64_t s = 0; s < nsamp; ++s) if (sa[s] >= 0) dp[sa[s] > sb[s] ? sa[s] : sb[s]] += 1;
    }
    return ne;
}

/* Tracked schedule: eliminate vertices from the counter-driven ready set,
 * picking a uniformly random ready vertex each time (splitmix64 stream
 * seeded by sched_seed; it decides only the schedule, never the numbers).
 * With check != 0, after every pivot the counters are recomputed from the
 * active multigraph and compared, and the ready set is checked to be
 * pairwise non-adjacent; mismatches are counted in F->violations. */
static uint64_t splitmix64(uint64_t *s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

int orc_factor_tracked_ac(int64_t n, const int64_t *colptr, const int32_t *rowind, const double *val,
                          const int32_t *ordering, int kind, uint64_t seed, uint64_t sys,
                          uint64_t sched_seed, int check, int ksplit, orc_factor **out)
{
    *out = NULL;
    if (ksplit < 0) return ORC_EINVAL;
    orc_state S;
    memset(&S, 0, sizeof S);
    S.ksamp = 1;
    S.ac = ksplit > 0;
    int rc = orc_ingest(n, colptr, rowind, val, ordering, kind, &S.L);
    if (rc) return rc;
    if (ksplit > 0) {
        rc = low_split(&S.L, ksplit);
        if (rc) { low_free(&S.L); return rc; }
    }
    rc = state_init(&S);
    int64_t nl = S.L.n;
    size_t nn = (size_t)(nl > 0 ? nl : 1);
    int32_t *dp = calloc(nn, sizeof(int32_t));
    int32_t *ready = malloc(sizeof(int32_t) * nn);
    char *done = calloc(nn, 1);
    int32_t *recount = calloc(nn, sizeof(int32_t));
    int32_t *enq = malloc(sizeof(int32_t) * (nn + 1));
    if (!dp || !ready || !done || !recount || !enq) rc = ORC_ENOMEM;
    int64_t nready = 0, violations = 0;
    if (!rc) {
        for (int64_t q = 0; q < S.L.colptr[nl]; ++q) dp[S.L.row[q]]++;   /* R8 */
        for (int64_t i = 0; i < nl; ++i) if (dp[i] == 0) ready[nready++] = (int32_t)i;
    }
    uint64_t sm = sched_seed;
    int64_t eliminated = 0;
    while (!rc && nready > 0) {
        int64_t pick = (int64_t)(splitmix64(&sm) % (uint64_t)nready);
        int32_t k = ready[pick];
        ready[pick] = ready[--nready];
        orc_step st;
        rc = state_eliminate(&S, k, seed, sys, &st);
        if (rc) break;
        done[k] = 1;
        eliminated++;
        int64_t ne = orc_dp_update(dp, st.ns, st.slo, st.shi, st.d, st.mrow, st.mmult, enq, 0);
        for (int64_t i = 0; i < ne; ++i) ready[nready++] = enq[i];
        step_free(&st);
        if (check) {
            /* recompute d_t(i): entries still waiting in active columns c */
            memset(recount, 0, sizeof(int32_t) * nn);
            for (int64_t c = 0; c < nl; ++c) {
                if (done[c]) continue;
                for (int64_t q = S.L.colptr[c]; q < S.L.colptr[c + 1]; ++q) recount[S.L.row[q]]++;
                for (int64_t q = 0; q < S.fill[c].cnt; ++q) recount[S.fill[c].row[q]]++;
            }
            for (int64_t i = 0; i < nl; ++i) if (!done[i] && recount[i] != dp[i]) violations++;
            /* ready pivots pairwise non-adjacent: no active column of a ready
             * vertex holds another ready vertex as a row */
            for (int64_t a = 0; a < nready; ++a) {
                int32_t c = ready[a];
                for (int64_t b = 0; b < nready; ++b) {
                    int32_t r = ready[b];
                    if (r <= c) continue;
                    for (int64_t q = S.L.colptr[c]; q < S.L.colptr[c + 1]; ++q) if (S.L.row[q] == r) violations++;
                    for (int64_t q = 0; q < S.fill[c].cnt; ++q) if (S.fill[c].row[q] == r) violations++;
                }
            }
            /* every ready vertex has counter zero */
            for (int64_t a = 0; a < nready; ++a) if (dp[ready[a]] != 0) violations++;
        }
    }
    if (!rc && eliminated != nl) violations += nl - eliminated;
    if (!rc) rc = state_to_factor(&S, out);
    if (!rc) (*out)->violations = violations;
    free(dp); free(ready); free(done); free(recount); free(enq);
    state_free(&S);
    return rc;
}

int orc_factor_tracked(int64_t n, const int64_t *colptr, const int32_t *rowind, const double *val,
                       const int32_t *ordering, int kind, uint64_t seed, uint64_t sys,
                       uint64_t sched_seed, int check, orc_factor **out)
{
    return orc_factor_tracked_ac(n, colptr, rowind, val, ordering, kind, seed, sys, sched_seed, check, 0, out);
}

/* ------------------------------------------------------------------------ */
/* Factor accessors.                                                         */
/* ------------------------------------------------------------------------ */
void orc_factor_dims(const orc_factor *F, int64_t *n, int64_t *nnz, int64_t stats[6])
{
    *n = F->n;
    *nnz = F->colptr[F->n];
    stats[0] = F->nnz_low_in; stats[1] = F->fill; stats[2] = F->nnz_all;
    stats[3] = F->max_gather; stats[4] = F->depth; stats[5] = F->violations;
}

void orc_factor_copy(const orc_factor *F, int64_t *colptr, int32_t *row, double *val, double *D)
{
    int64_t nnz = F->colptr[F->n];
    memcpy(colptr, F->colptr, sizeof(int64_t) * (size_t)(F->n + 1));
    if (nnz) { memcpy(row, F->row, sizeof(int32_t) * (size_t)nnz); memcpy(val, F->val, sizeof(double) * (size_t)nnz); }
    if (F->n) memcpy(D, F->D, sizeof(double) * (size_t)F->n);
}

void orc_factor_free(orc_factor *F)
{
    if (!F) return;
    free(F->colptr); free(F->row); free(F->val); free(F->D); free(F);
}

/* One pivot on its own (for the sampling tests): gathered (rows, w) of g
 * entries in, merged neighbours / F values / sampled edges out.  Output
 * arrays need room for g entries.  Returns d via *d_out and D via *D_out. */
int orc_eliminate_one(int64_t g, const int32_t *rows, const double *w, uint64_t seed, uint64_t k,
                      uint64_t sys, int64_t *d_out, double *D_out, int32_t *mrow, double *mw,
                      int32_t *mmult, double *fval, int32_t *slo, int32_t *shi, double *sc,
                      int64_t *spick)
{
    orc_step st = { 0, 0.0, mrow, mw, mmult, fval, slo, shi, sc, spick, 0 };
    int rc = orc_eliminate(g, rows, w, seed, k, sys, &st);
    *d_out = st.d; *D_out = st.D;
    return rc;
}

/* As orc_eliminate_one with ksamp samples per slot; sampled-edge arrays need
 * room for ksamp * g entries (sample q of slot p at q*(d-1) + p-1). */
int orc_eliminate_one_k(int64_t g, const int32_t *rows, const double *w, uint64_t seed, uint64_t k,
                        uint64_t sys, int ksamp, int64_t *d_out, double *D_out, int32_t *mrow, double *mw,
                        int32_t *mmult, double *fval, int32_t *slo, int32_t *shi, double *sc, int64_t *spick)
{
    if (ksamp < 1) return ORC_EINVAL;
    orc_step st = { 0, 0.0, mrow, mw, mmult, fval, slo, shi, sc, spick, 0 };
    int rc = orc_eliminate_k(g, rows, w, seed, k, sys, ksamp, &st);
    *d_out = st.d; *D_out = st.D;
    return rc;
}

/* One AC(k) pivot (orc_eliminate_ac) on gathered entries; the slot arrays
 * need room for g entries; *ns_out receives the slot count (g - 1). */
int orc_eliminate_one_ac(int64_t g, const int32_t *rows, const double *w, uint64_t seed, uint64_t k,
                         uint64_t sys, int64_t *d_out, double *D_out, int64_t *ns_out, int32_t *mrow, double *mw,
                         int32_t *mmult, double *fval, int32_t *slo, int32_t *shi, double *sc, int64_t *spick)
{
    orc_step st = { 0, 0.0, mrow, mw, mmult, fval, slo, shi, sc, spick, 0 };
    int rc = orc_eliminate_ac(g, rows, w, seed, k, sys, &st);
    *d_out = st.d; *D_out = st.D; *ns_out = st.ns;
    return rc;
}

/* Strict lower CSC as ingested (for tests of the ingest step). */
int orc_ingest_dims(int64_t n, const int64_t *colptr, const int32_t *rowind, const double *val,
                    const int32_t *ordering, int kind, int64_t *nl, int64_t *nnz, int *ground)
{
    orc_low L;
    int rc = orc_ingest(n, colptr, rowind, val, ordering, kind, &L);
    if (rc) return rc;
    *nl = L.n; *nnz = L.colptr[L.n]; *ground = L.has_ground;
    low_free(&L);
    return ORC_OK;
}

int orc_ingest_copy(int64_t n, const int64_t *colptr, const int32_t *rowind, const double *val,
                    const int32_t *ordering, int kind, int64_t *cp, int32_t *row, double *w)
{
    orc_low L;
    int rc = orc_ingest(n, colptr, rowind, val, ordering, kind, &L);
    if (rc) return rc;
    memcpy(cp, L.colptr, sizeof(int64_t) * (size_t)(L.n + 1));
    int64_t m = L.colptr[L.n];
    if (m) { memcpy(row, L.row, sizeof(int32_t) * (size_t)m); memcpy(w, L.w, sizeof(double) * (size_t)m); }
    low_free(&L);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Preconditioner apply and PCG.                                             */
/* ------------------------------------------------------------------------ */

/* z = P^T F^{-T} D^+ F^{-1} P r, where (P r)[k] = r[ordering[k]].  F is the
 * strict-lower CSC of a unit lower-triangular matrix in label space. */
void orc_precond_apply(int64_t n, const int64_t *fcp, const int32_t *frow, const double *fval,
                       const double *D, const int32_t *ordering, const double *r, double *z,
                       double *work)
{
    double *y = work;
    for (int64_t k = 0; k < n; ++k) y[k] = r[ordering ? ordering[k] : k];
    for (int64_t k = 0; k < n; ++k)                       /* y <- F^{-1} y */
        for (int64_t q = fcp[k]; q < fcp[k + 1]; ++q) y[frow[q]] = y[frow[q]] - fval[q] * y[k];
    for (int64_t k = 0; k < n; ++k) y[k] = D[k] > 0.0 ? y[k] / D[k] : 0.0;
    for (int64_t k = n - 1; k >= 0; --k) {                /* y <- F^{-T} y */
        double s = y[k];
        for (int64_t q = fcp[k]; q < fcp[k + 1]; ++q) s = s - fval[q] * y[frow[q]];
        y[k] = s;
    }
    for (int64_t k = 0; k < n; ++k) z[ordering ? ordering[k] : k] = y[k];
}

/* ------------------------------------------------------------------------ */
/* Mixed precision: the factor stored and applied in FP32 inside FP64 PCG.   */
/* ------------------------------------------------------------------------ */
/* The paper runs the whole method in FP64.  The mixed form keeps the
 * elimination and PCG's recurrences in FP64 and applies the factor in FP32,
 * read as follows (the same reading as the FP64 apply above otherwise):
 *   M1  F32 = RN32(F) entry by entry (round to nearest even); the right-hand
 *       side enters the forward solve as RN32(r).
 *   M2  forward solve in dot form: y_j = RN32(r_j) - t_j, where t_j is the
 *       FP32 sum of the FP32 products F32(j,c) * y_c over c < j (every
 *       product and every addition rounded to FP32).
 *   M3  scale by D^+: D^+_k = 1 / D_k in FP64 (0 where D_k = 0); the scaled
 *       unknown is s_k = RN32(y_k * D^+_k) with the product formed in FP64.
 *   M4  backward solve in dot form: z_j = s_j - (FP32 sum of the FP32
 *       products F32(i,j) * z_i over i > j).
 *   M5  z is returned widened to FP64 (exact).
 * The order of the FP32 sums in M2/M4 is not part of the reading: any order
 * is a correct evaluation (this file adds in ascending index order).  The
 * componentwise bound computed alongside holds for every order, so another
 * evaluation is compared with this one through it; when every sum has at
 * most two terms all orders give the same bits.
 *
 * Error bound (running error analysis, u = 2^-24, gamma_m = m u/(1 - m u)):
 * with F = I + N and exact FP64 data (F, D, r), the computed forward
 * unknowns satisfy |y^_j - (r_j - sum_c F_jc y^_c)| <= rho_j with
 *   rho_j = gamma_{m_j+2} (|r_j| + |y^_j| + sum_c |F_jc| |y^_c|),
 * m_j the row length; so |y^ - y| <= |F^{-1}| rho <= (I - |N|)^{-1} rho
 * (|F^{-1}| = |sum_k (-N)^k| <= sum_k |N|^k, N nilpotent).  The scale adds
 * D^+_k (u + 2^-51) |y^_k|; the backward solve adds, through
 * (I - |N|^T)^{-1}, rho'_j = gamma_{m'_j+1} (|z^_j| + sum_i |F_ij| |z^_i|).
 * Both positive triangular solves are done here in FP64 and the result is
 * inflated by 2^-40 relative to cover their own rounding. */
static double orc_gamma32(int64_t m)
{
    const double mu = (double)m * 0x1.0p-24;
    return mu / (1.0 - mu);
}

int orc_precond_apply32(int64_t n, const int64_t *fcp, const int32_t *frow, const double *fval,
                        const double *D, const int32_t *ordering, const double *r, double *z, double *bound)
{
    size_t nn = (size_t)(n > 0 ? n : 1);
    int64_t nnz = fcp[n];
    size_t mm = (size_t)(nnz > 0 ? nnz : 1);
    int64_t *rp = calloc(nn + 1, sizeof(int64_t)), *next = malloc(sizeof(int64_t) * nn);
    int32_t *rc = malloc(sizeof(int32_t) * mm);
    float *cv = malloc(sizeof(float) * mm), *rv = malloc(sizeof(float) * mm);
    double *rv64 = malloc(sizeof(double) * mm);
    float *y = malloc(sizeof(float) * nn), *s = malloc(sizeof(float) * nn), *zz = malloc(sizeof(float) * nn);
    double *dplus = malloc(sizeof(double) * nn);
    if (!rp || !next || !rc || !cv || !rv || !rv64 || !y || !s || !zz || !dplus) {
        free(rp); free(next); free(rc); free(cv); free(rv); free(rv64); free(y); free(s); free(zz); free(dplus);
        return ORC_ENOMEM;
    }
    for (int64_t q = 0; q < nnz; ++q) cv[q] = (float)fval[q];                       /* M1 */
    /* rows of F (the forward solve's dot products), columns ascending */
    for (int64_t q = 0; q < nnz; ++q) rp[frow[q] + 1]++;
    for (int64_t j = 0; j < n; ++j) rp[j + 1] += rp[j];
    for (int64_t j = 0; j < n; ++j) next[j] = rp[j];
    for (int64_t k = 0; k < n; ++k)
        for (int64_t q = fcp[k]; q < fcp[k + 1]; ++q) {
            int64_t at = next[frow[q]]++;
            rc[at] = (int32_t)k; rv[at] = cv[q]; rv64[at] = fval[q];
        }
    for (int64_t j = 0; j < n; ++j) {                                               /* M2 */
        float t = 0.0f;
        for (int64_t a = rp[j]; a < rp[j + 1]; ++a) {
            float prod = rv[a] * y[rc[a]];
            t = t + prod;
        }
        float rj = (float)r[ordering ? ordering[j] : j];
        y[j] = rj - t;
    }
    for (int64_t k = 0; k < n; ++k) {                                               /* M3 */
        dplus[k] = D[k] > 0.0 ? 1.0 / D[k] : 0.0;
        s[k] = (float)((double)y[k] * dplus[k]);
    }
    for (int64_t j = n - 1; j >= 0; --j) {                                          /* M4 */
        float t = 0.0f;
        for (int64_t q = fcp[j]; q < fcp[j + 1]; ++q) {
            float prod = cv[q] * zz[frow[q]];
            t = t + prod;
        }
        zz[j] = s[j] - t;
    }
    for (int64_t k = 0; k < n; ++k) z[ordering ? ordering[k] : k] = (double)zz[k];  /* M5 */

    if (bound) {
        double *ey = malloc(sizeof(double) * nn), *ez = malloc(sizeof(double) * nn);
        if (!ey || !ez) {
            free(ey); free(ez);
            free(rp); free(next); free(rc); free(cv); free(rv); free(rv64); free(y); free(s); free(zz); free(dplus);
            return ORC_ENOMEM;
        }
        for (int64_t j = 0; j < n; ++j) {
            double fy = 0.0, fe = 0.0;
            for (int64_t a = rp[j]; a < rp[j + 1]; ++a) {
                fy += fabs(rv64[a]) * fabs((double)y[rc[a]]);
                fe += fabs(rv64[a]) * ey[rc[a]];
            }
            double rj = fabs(r[ordering ? ordering[j] : j]);
            double rho = orc_gamma32(rp[j + 1] - rp[j] + 2) * (rj + fabs((double)y[j]) + fy);
            ey[j] = rho + fe;
        }
        for (int64_t j = n - 1; j >= 0; --j) {
            double es = dplus[j] * (ey[j] + (0x1.0p-24 + 0x1.0p-51) * fabs((double)y[j]));
            double fz = 0.0, fe = 0.0;
            for (int64_t q = fcp[j]; q < fcp[j + 1]; ++q) {
                fz += fabs(fval[q]) * fabs((double)zz[frow[q]]);
                fe += fabs(fval[q]) * ez[frow[q]];
            }
            double rho = orc_gamma32(fcp[j + 1] - fcp[j] + 1) * (fabs((double)zz[j]) + fz);
            ez[j] = es + rho + fe;
        }
        for (int64_t k = 0; k < n; ++k) bound[ordering ? ordering[k] : k] = ez[k] * (1.0 + 0x1.0p-40);
        free(ey); free(ez);
    }
    free(rp); free(next); free(rc); free(cv); free(rv); free(rv64); free(y); free(s); free(zz); free(dplus);
    return ORC_OK;
}

static void spmv(int64_t n, const int64_t *cp, const int32_t *ri, const double *v, const double *x, double *y)
{
    /* L is symmetric, so its CSC is also its CSR: y_i = sum over column i. */
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t q = cp[i]; q < cp[i + 1]; ++q) s = s + v[q] * x[ri[q]];
        y[i] = s;
    }
}

static double dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s = s + a[i] * b[i];
    return s;
}

/* PCG for L x = b from x0 = 0.  Stops when the recurrence residual satisfies
 * ||r|| <= tol ||b|| AND the recomputed true residual ||b - L x|| <= tol ||b||,
 * or after maxit iterations.  tol <= 0 runs exactly maxit iterations.
 * Returns iterations through *iters and the true relative residual. */
static int apply_prec(int prec, int64_t n, const int64_t *fcp, const int32_t *frow, const double *fval,
                      const double *D, const int32_t *ordering, const double *r, double *z, double *work)
{
    if (prec == 32) return orc_precond_apply32(n, fcp, frow, fval, D, ordering, r, z, NULL);
    orc_precond_apply(n, fcp, frow, fval, D, ordering, r, z, work);
    return ORC_OK;
}

/* prec = 64: the FP64 apply; prec = 32: the mixed form (M1-M5 above) inside
 * the same FP64 recurrences. */
int orc_pcg_prec(int64_t n, const int64_t *cp, const int32_t *ri, const double *v,
                 const int64_t *fcp, const int32_t *frow, const double *fval, const double *D,
                 const int32_t *ordering, const double *b, double tol, int32_t maxit, int prec,
                 double *x, int32_t *iters, double *true_relres)
{
    if (prec != 32 && prec != 64) return ORC_EINVAL;
    size_t nn = (size_t)(n > 0 ? n : 1);
    double *r = malloc(sizeof(double) * nn), *z = malloc(sizeof(double) * nn);
    double *p = malloc(sizeof(double) * nn), *q = malloc(sizeof(double) * nn);
    double *work = malloc(sizeof(double) * nn);
    if (!r || !z || !p || !q || !work) { free(r); free(z); free(p); free(q); free(work); return ORC_ENOMEM; }
    double nb = sqrt(dot(n, b, b));
    for (int64_t i = 0; i < n; ++i) { x[i] = 0.0; r[i] = b[i]; }
    int32_t it = 0;
    double relres = nb > 0.0 ? 1.0 : 0.0;
    if (nb > 0.0) {
        if (apply_prec(prec, n, fcp, frow, fval, D, ordering, r, z, work)) {
            free(r); free(z); free(p); free(q); free(work); return ORC_ENOMEM;
        }
        for (int64_t i = 0; i < n; ++i) p[i] = z[i];
        double rz = dot(n, r, z);
        while (it < maxit) {
            spmv(n, cp, ri, v, p, q);
            double alpha = rz / dot(n, p, q);
            for (int64_t i = 0; i < n; ++i) x[i] = x[i] + alpha * p[i];
            for (int64_t i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];
            ++it;
            if (tol > 0.0 && sqrt(dot(n, r, r)) <= tol * nb) {
                spmv(n, cp, ri, v, x, q);
                for (int64_t i = 0; i < n; ++i) q[i] = b[i] - q[i];
                if (sqrt(dot(n, q, q)) <= tol * nb) break;
            }
            if (apply_prec(prec, n, fcp, frow, fval, D, ordering, r, z, work)) {
                free(r); free(z); free(p); free(q); free(work); return ORC_ENOMEM;
            }
            double rz2 = dot(n, r, z);
            double beta = rz2 / rz;
            rz = rz2;
            for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
        }
        spmv(n, cp, ri, v, x, q);
        for (int64_t i = 0; i < n; ++i) q[i] = b[i] - q[i];
        relres = sqrt(dot(n, q, q)) / nb;
    }
    *iters = it;
    *true_relres = relres;
    free(r); free(z); free(p); free(q); free(work);
    return ORC_OK;
}

int orc_pcg(int64_t n, const int64_t *cp, const int32_t *ri, const double *v,
            const int64_t *fcp, const int32_t *frow, const double *fval, const double *D,
            const int32_t *ordering, const double *b, double tol, int32_t maxit,
            double *x, int32_t *iters, double *true_relres)
{
    return orc_pcg_prec(n, cp, ri, v, fcp, frow, fval, D, ordering, b, tol, maxit, 64, x, iters, true_relres);
}
