/*
 * CPU oracle for the quantised layered LDPC reconciliation decoder.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the bench's
 * CPU-baseline leg load this file's library.  It shares no code, header or
 * table with the CUDA path and never calls it.
 *
 * Plain scalar C, one frame at a time, written so that each step can be
 * checked against the paper by eye:
 *   - QC-LDPC lifting of a base matrix (section 4.1);
 *   - layered schedule with only E_j and L_ij stored, L_ji formed on the fly
 *     (section 2, Eqs. 8 and 9);
 *   - check node: sign product (Eq. 1) times the syndrome sign, magnitude by
 *     repeated box-plus (Eq. 7) with the integer table tau of Algorithm 1
 *     (section 3.2);
 *   - variable node: saturation-oriented update of Algorithm 2 (section 3.3);
 *   - stopping test: all parity checks tested with the latest E_j at the end
 *     of each iteration (section 2); optionally a stall window K that also
 *     stops, as a failure, a frame whose count of unsatisfied checks has set
 *     no new minimum for K iterations (not in the paper; off by default).
 * Readings where the paper is silent (fold order, L_ji width, syndrome sign,
 * degree-1 rows, LLR scale, offset tables) are the ones listed in the design
 * notes; each is marked "Reading" below.
 *
 * Circulant convention: base entry s >= 0 at block (i, k) connects row r of
 * block row i to variable node k*Z + ((r + s) mod Z).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORC_E_MAX 127 /* Algorithm 2: predefined maximum magnitude for 8 bits */

/* ---------------------------------------------------------------- helpers */

static int sat8(int x) { return x > 127 ? 127 : (x < -127 ? -127 : x); }
static int sgn(int x) { return x < 0 ? -1 : 1; } /* Reading: sign of 0 is + */
static int imin(int a, int b) { return a < b ? a : b; }
static int imax(int a, int b) { return a > b ? a : b; }

/* Algorithm 1 (section 3.2): integer box-plus table tau(p, q). */
int orc_tau(int p, int q, int msg_max) {
    int a = imin(p, msg_max);
    int b = imin(q, msg_max);
    int g = imax(a, b);
    int l = imin(a, b);
    int d = g - l;
    if (l > 2) return l - (d < 2) - (d < 6);
    return imax(l - (d < 4), 0);
}

/* Reading (offset tables): m' = clamp(((m*s + 8) >> 4) - o, 0, msg_max).
 * s = 16, o = 0 is the identity, i.e. the plain decoder of the paper. */
static int apply_table(int m, int s, int o, int msg_max) {
    int x = ((m * s + 8) >> 4) - o;
    return x < 0 ? 0 : (x > msg_max ? msg_max : x);
}

/* Algorithm 2 (section 3.3): update E_j only while |E_j| != E_max. */
int orc_vn_update(int e_old, int l_ji, int l_ij_new) {
    if (abs(e_old) != ORC_E_MAX) return sat8(l_ji + l_ij_new);
    return e_old;
}

/* ------------------------------------------------------ code expansion */

typedef struct {
    int Mb, Nb, Z, n, m;
    int64_t edges;
    int32_t* row_ptr; /* m + 1 */
    int32_t* vn;      /* edges: VN index, rows in layer-major order, ascending VN within a row */
} orc_graph;

static int build_graph(const int32_t* base, int Mb, int Nb, int Z, orc_graph* g) {
    g->Mb = Mb; g->Nb = Nb; g->Z = Z; g->n = Nb * Z; g->m = Mb * Z;
    int64_t e = 0;
    for (int i = 0; i < Mb * Nb; i++) e += base[i] >= 0;
    g->edges = e * Z;
    g->row_ptr = (int32_t*)malloc(sizeof(int32_t) * (size_t)(g->m + 1));
    g->vn = (int32_t*)malloc(sizeof(int32_t) * (size_t)(g->edges ? g->edges : 1));
    if (!g->row_ptr || !g->vn) return -1;
    int64_t pos = 0;
    for (int i = 0; i < Mb; i++) {
        for (int r = 0; r < Z; r++) {
            g->row_ptr[i * Z + r] = (int32_t)pos;
            for (int k = 0; k < Nb; k++) {
                int s = base[i * Nb + k];
                if (s < 0) continue;
                g->vn[pos++] = k * Z + (r + s) % Z;
            }
        }
    }
    g->row_ptr[g->m] = (int32_t)pos;
    return 0;
}

static void free_graph(orc_graph* g) { free(g->row_ptr); free(g->vn); }

int64_t orc_edge_count(const int32_t* base, int Mb, int Nb, int Z) {
    int64_t e = 0;
    for (int i = 0; i < Mb * Nb; i++) e += base[i] >= 0;
    return e * Z;
}

/* Row lists of H, for tests: row_ptr[m+1], vn[edges]. */
int orc_expand(const int32_t* base, int Mb, int Nb, int Z, int32_t* row_ptr, int32_t* vn) {
    orc_graph g;
    if (build_graph(base, Mb, Nb, Z, &g)) return -1;
    memcpy(row_ptr, g.row_ptr, sizeof(int32_t) * (size_t)(g.m + 1));
    memcpy(vn, g.vn, sizeof(int32_t) * (size_t)g.edges);
    free_graph(&g);
    return 0;
}

/* ----------------------------------------------------------- syndrome */

static void syndrome_one(const orc_graph* g, const uint8_t* bits, uint8_t* syn) {
    for (int c = 0; c < g->m; c++) {
        int par = 0;
        for (int32_t e = g->row_ptr[c]; e < g->row_ptr[c + 1]; e++) par ^= bits[g->vn[e]] & 1;
        syn[c] = (uint8_t)par;
    }
}

/* s = H x (mod 2) for a batch of unpacked bit vectors [batch][n] -> [batch][m]. */
int orc_syndrome(const int32_t* base, int Mb, int Nb, int Z, const uint8_t* bits, int batch, uint8_t* syn) {
    orc_graph g;
    if (build_graph(base, Mb, Nb, Z, &g)) return -1;
    for (int f = 0; f < batch; f++) syndrome_one(&g, bits + (size_t)f * g.n, syn + (size_t)f * g.m);
    free_graph(&g);
    return 0;
}

/* -------------------------------------------------- channel LLRs (3.1) */

/* Reading (LLR scale): channel LLR magnitude = round-half-away(ln((1-p)/p) * scale),
 * clamped to 127; sign + for a received 0.  Punctured positions get 0,
 * shortened positions +-127 by their known value. */
int orc_llr_magnitude(double p, double scale) {
    double x = log((1.0 - p) / p) * scale;
    long r = lround(x);
    if (r > 127) r = 127;
    if (r < -127) r = -127;
    return (int)r;
}

/* state[j]: 0 = key bit, 1 = punctured, 2 = shortened (known value in known[j]). */
void orc_llr_frame(const uint8_t* y, const uint8_t* state, const uint8_t* known, double p, double scale,
                   int n, int8_t* llr) {
    int mag = orc_llr_magnitude(p, scale);
    for (int j = 0; j < n; j++) {
        int st = state ? state[j] : 0;
        if (st == 1) llr[j] = 0;
        else if (st == 2) llr[j] = (int8_t)(known[j] ? -ORC_E_MAX : ORC_E_MAX);
        else llr[j] = (int8_t)(y[j] ? -mag : mag);
    }
}

/* ------------------------------------------------- check-node magnitudes */

/* fold_mode 0 (normative reading of Eq. 7): for edge k, the box-plus of all
 * other magnitudes in ascending VN order, realised as
 *   F_k = tau(F_{k-1}, a_k) (left fold), B_k = tau(a_k, B_{k+1}) (right fold),
 *   m_k = tau(F_{k-1}, B_{k+1}), m_0 = B_1, m_{d-1} = F_{d-2}.
 * fold_mode 1: Eq. 7 taken literally per edge, a right-nested fold of the
 *   other d-1 magnitudes in ascending order (diagnostic variant).
 * fold_mode 2: tau replaced by min (textbook min-sum), for pinning.
 * Reading (degree 1): the box-plus over no operand is +inf -> msg_max. */
static int tau_m(int p, int q, int msg_max, int mode) {
    if (mode == 2) return imin(imin(p, q), msg_max);
    return orc_tau(p, q, msg_max);
}

void orc_cn_magnitudes(const int* a, int d, int msg_max, int fold_mode, int* m) {
    if (d <= 0) return;
    if (d == 1) { m[0] = msg_max; return; }
    if (fold_mode == 1) {
        for (int k = 0; k < d; k++) {
            int acc = -1;
            for (int q = d - 1; q >= 0; q--) {
                if (q == k) continue;
                acc = acc < 0 ? imin(a[q], msg_max) : tau_m(a[q], acc, msg_max, 0);
            }
            m[k] = acc;
        }
        return;
    }
    int* F = (int*)malloc(sizeof(int) * (size_t)d);
    int* B = (int*)malloc(sizeof(int) * (size_t)d);
    F[0] = imin(a[0], msg_max);
    for (int k = 1; k < d; k++) F[k] = tau_m(F[k - 1], a[k], msg_max, fold_mode);
    B[d - 1] = imin(a[d - 1], msg_max);
    for (int k = d - 2; k >= 0; k--) B[k] = tau_m(a[k], B[k + 1], msg_max, fold_mode);
    m[0] = B[1];
    m[d - 1] = F[d - 2];
    for (int k = 1; k < d - 1; k++) m[k] = tau_m(F[k - 1], B[k + 1], msg_max, fold_mode);
    free(F);
    free(B);
}

/* ------------------------------------------------------------ decoding */

typedef struct {
    int max_iter, msg_max, fold_mode;
    const uint8_t* scale_q4; /* [max_iter][Mb] or NULL */
    const int8_t* offset_q;  /* [max_iter][Mb] or NULL */
    int stall;               /* stall window K, 0 = off */
} orc_opts;

static int row_parity_ok(const orc_graph* g, const int8_t* E, const uint8_t* syn) {
    for (int c = 0; c < g->m; c++) {
        int par = 0;
        for (int32_t e = g->row_ptr[c]; e < g->row_ptr[c + 1]; e++) par ^= E[g->vn[e]] < 0;
        if (par != (syn[c] & 1)) return 0;
    }
    return 1;
}

/* Number of parity checks the hard decisions E < 0 leave unsatisfied. */
static int unsatisfied_checks(const orc_graph* g, const int8_t* E, const uint8_t* syn) {
    int u = 0;
    for (int c = 0; c < g->m; c++) {
        int par = 0;
        for (int32_t e = g->row_ptr[c]; e < g->row_ptr[c + 1]; e++) par ^= E[g->vn[e]] < 0;
        u += par != (syn[c] & 1);
    }
    return u;
}

/* One frame: llr[n], syn[m] (unpacked) -> bits[n] (unpacked), iterations, ok. */
static void decode_one(const orc_graph* g, const orc_opts* o, const int8_t* llr, const uint8_t* syn,
                       int8_t* E, int8_t* L, int* v, int* a, int* mag, uint8_t* bits, int32_t* iters,
                       uint8_t* ok) {
    for (int j = 0; j < g->n; j++) E[j] = llr[j];
    memset(L, 0, (size_t)g->edges);
    int done = 0, stalled = 0, t = 0;
    int u_best = 0x7FFFFFFF, t_best = 0; /* stall rule: fewest unsatisfied checks so far, first reached at t_best */
    for (t = 1; t <= o->max_iter; t++) {
        for (int i = 0; i < g->Mb; i++) {            /* Reading: one block row = one layer */
            for (int r = 0; r < g->Z; r++) {         /* rows of a layer share no VN */
                int c = i * g->Z + r;
                int32_t e0 = g->row_ptr[c];
                int d = g->row_ptr[c + 1] - e0;
                if (d == 0) continue;
                int S = (syn[c] & 1) ? -1 : 1;       /* Reading: syndrome flips the CN sign */
                for (int k = 0; k < d; k++) {
                    int j = g->vn[e0 + k];
                    v[k] = sat8(E[j] - L[e0 + k]);   /* Eq. 8; Reading: L_ji saturated to int8 */
                    a[k] = imin(abs(v[k]), o->msg_max);
                    S *= sgn(v[k]);                  /* Eq. 1 */
                }
                orc_cn_magnitudes(a, d, o->msg_max, o->fold_mode, mag);
                for (int k = 0; k < d; k++) {
                    int mk = mag[k];
                    if (o->scale_q4 || o->offset_q) {
                        int s = o->scale_q4 ? o->scale_q4[(t - 1) * g->Mb + i] : 16;
                        int off = o->offset_q ? o->offset_q[(t - 1) * g->Mb + i] : 0;
                        mk = apply_table(mk, s, off, o->msg_max);
                    }
                    int lnew = S * sgn(v[k]) * mk;  /* exclude the edge's own sign */
                    int j = g->vn[e0 + k];
                    E[j] = (int8_t)orc_vn_update(E[j], v[k], lnew); /* Eq. 9 under Algorithm 2 */
                    L[e0 + k] = (int8_t)lnew;
                }
            }
        }
        /* stopping test at the end of the iteration (section 2) */
        if (o->stall > 0) {
            /* Stall rule (not in the paper; off unless asked for): a frame whose
             * count of unsatisfied checks has set no new minimum for K
             * iterations stops as a failure. */
            int u = unsatisfied_checks(g, E, syn);
            if (u == 0) { done = 1; break; }
            if (u < u_best) { u_best = u; t_best = t; }
            else if (t - t_best >= o->stall) { stalled = 1; break; }
        } else if (row_parity_ok(g, E, syn)) {
            done = 1;
            break;
        }
    }
    for (int j = 0; j < g->n; j++) bits[j] = E[j] < 0; /* Reading: E = 0 decides 0 */
    *iters = (done || stalled) ? t : o->max_iter;
    *ok = (uint8_t)done;
}

typedef struct {
    const orc_graph* g;
    const orc_opts* o;
    const int8_t* llr;
    const uint8_t* syn;
    uint8_t* bits;
    int32_t* iters;
    uint8_t* ok;
    int batch, next;
    pthread_mutex_t* mu;
} orc_job;

static void* worker(void* arg) {
    orc_job* J = (orc_job*)arg;
    const orc_graph* g = J->g;
    int dmax = 0;
    for (int c = 0; c < g->m; c++) dmax = imax(dmax, g->row_ptr[c + 1] - g->row_ptr[c]);
    int8_t* E = (int8_t*)malloc((size_t)g->n);
    int8_t* L = (int8_t*)malloc((size_t)(g->edges ? g->edges : 1));
    int* v = (int*)malloc(sizeof(int) * (size_t)(dmax + 1));
    int* a = (int*)malloc(sizeof(int) * (size_t)(dmax + 1));
    int* mg = (int*)malloc(sizeof(int) * (size_t)(dmax + 1));
    for (;;) {
        pthread_mutex_lock(J->mu);
        int f = J->next++;
        pthread_mutex_unlock(J->mu);
        if (f >= J->batch) break;
        decode_one(g, J->o, J->llr + (size_t)f * g->n, J->syn + (size_t)f * g->m, E, L, v, a, mg,
                   J->bits + (size_t)f * g->n, J->iters + f, J->ok + f);
    }
    free(E); free(L); free(v); free(a); free(mg);
    return NULL;
}

int orc_num_cores(void) {
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    return c > 0 ? (int)c : 1;
}

/* Decode a batch: llr[batch][n] int8, syn[batch][m] unpacked -> bits[batch][n]
 * unpacked, iters[batch], ok[batch].  stall = K > 0 enables the stall rule.
 * threads <= 0 uses every online core.
 * Returns the number of threads used, or a negative value on error. */
int orc_decode_batch(const int32_t* base, int Mb, int Nb, int Z, const int8_t* llr, const uint8_t* syn,
                     int batch, int max_iter, int msg_max, int fold_mode, const uint8_t* scale_q4,
                     const int8_t* offset_q, int stall, uint8_t* bits, int32_t* iters, uint8_t* ok, int threads) {
    orc_graph g;
    if (Mb <= 0 || Nb <= 0 || Z <= 0 || batch < 0 || max_iter < 1 || stall < 0) return -1;
    if (build_graph(base, Mb, Nb, Z, &g)) return -2;
    orc_opts o = {max_iter, msg_max, fold_mode, scale_q4, offset_q, stall};
    if (threads <= 0) threads = orc_num_cores();
    if (threads > batch) threads = batch > 0 ? batch : 1;
    pthread_mutex_t mu = PTHREAD_MUTEX_INITIALIZER;
    orc_job J = {&g, &o, llr, syn, bits, iters, ok, batch, 0, &mu};
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)threads);
    for (int k = 0; k < threads; k++) pthread_create(&th[k], NULL, worker, &J);
    for (int k = 0; k < threads; k++) pthread_join(th[k], NULL);
    free(th);
    free_graph(&g);
    return threads;
}
