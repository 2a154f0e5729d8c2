/*
 * chp_oracle.c -- plain, unpacked CPU stabilizer-tableau simulator.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline / reference legs of bench.py load this file's library.  The
 * product path (the CUDA library) never calls it, and the two share no code.
 *
 * What it computes: the Clifford backend of Qibo 0.2.9 (arXiv:2408.00384,
 * section "Simulation of Clifford circuits") is built on the phase-space
 * (stabilizer tableau) formalism of Aaronson & Gottesman, "Improved
 * simulation of stabilizer circuits", PRA 70, 052328 (2004).  This file
 * restates that algorithm (AG Sec. III) one bit per byte, with no packing,
 * blocking or fusion:
 *
 *   rows 0..n-1   destabilizers, rows n..2n-1 stabilizers, row 2n scratch;
 *   row i is the Pauli (-1)^r_i  (x) P(x_ij, z_ij),
 *   P(0,0)=I, P(1,0)=X, P(1,1)=Y, P(0,1)=Z.
 *
 * Gates: CNOT, H and phase S are AG's three update rules.  Every other gate
 * is built from them as a product of conjugations (Z = S S, X = H Z H,
 * Y = X Z up to a global phase, S^dagger = S S S, CZ = H_b CNOT H_b,
 * SWAP = three CNOTs), so only AG's rules are trusted here.
 *
 * Measurement of Z_a: AG's two cases.  The random outcome bit comes from
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11), written here from that paper's definition.
 *
 * Readings where the algorithm leaves a choice:
 *  - pivot p is the smallest stabilizer row with x_pa = 1;
 *  - the destabilizer row p-n is not passed through rowsum, because AG replace
 *    it by row p right afterwards (its rowsum would be an anticommuting
 *    product that is discarded);
 *  - the k-th measurement op of a (circuit, shot) draws Philox counter
 *    (k, shot, circuit_id lo, circuit_id hi) under key (seed lo, seed hi) and
 *    uses bit 0 of output word 0, whether or not the outcome is random;
 *  - MZR = measure, then apply X_a when the outcome is 1;
 *  - MX and MY measure X_a and Y_a by conjugation: X = H Z H, and
 *    Y = (H S^dagger)^dagger Z (H S^dagger), i.e. S^dagger, H, measure Z,
 *    H, S; they draw from the same measurement counter as MZ;
 *  - noise op j (DEPOL1, XERR, ZERR; counted per tableau from 0 in program
 *    order) draws Philox counter (j, shot, circuit_id lo, circuit_id hi) under
 *    key (seed lo, seed hi XOR 0x4E4F4953); it fires when word 0 shifted
 *    right by 4 is below the 28-bit probability field, and DEPOL1 then takes
 *    X, Y or Z by floor(word 1 * 3 / 2^32).
 *
 * Threads (orc_set_threads): AG's gate rules update every row from that
 * row's own bits, and the rowsums of a random-outcome measurement each write
 * a different target row while reading only the pivot row.  Those two loops
 * over rows may therefore be split into contiguous shares, one per thread,
 * with results identical to the one-thread run; nothing else is reordered.
 * The one-thread mode is the default.
 *
 * Parity pins: gate rules and g against explicit Pauli matrices; the whole
 * simulator against brute-force state vectors (n <= 10), known states and the
 * symplectic invariant; Philox against the Random123 known-answer vectors;
 * every thread count against the one-thread run.
 */
#include <pthread.h>
#include <sched.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ERANGE (-2)
#define ORC_ENOMEM (-3)
#define ORC_EPHASE (-8) /* rowsum met an odd exponent: not a commuting product */

typedef struct orc_pool orc_pool;

typedef struct {
  int32_t n;
  int64_t rows; /* 2n + 1: the last row is AG's scratch row */
  uint8_t *x, *z, *r;
  uint8_t *spare;         /* rows * n bytes: the target of a change of storage order */
  int64_t srow, scol;     /* element (i, j) of x and z sits at [i * srow + j * scol] */
  int64_t row_gates;      /* gate rules run since the last measurement in row-major order */
  uint64_t noise_counter; /* next noise-op index */
  orc_pool *pool;         /* worker threads, or NULL for one thread */
} orc_tab;

/* storage: one byte per bit, element (row i, qubit j) at
 * [i * srow + j * scol].  A gate reads and writes one or two qubits' columns
 * of every row, a rowsum whole rows; the tableau is kept row-major (srow n,
 * scol 1) while measurements run and qubit-major (srow 1, scol rows) while
 * gates run, switching to qubit-major once more than n/16 + 16 gate rules
 * follow a measurement (so that a reset's X between measurements does not
 * reorder twice).  Every access goes through these macros, so results do not
 * depend on the order. */
#define XB(t, i, j) ((t)->x[(int64_t)(i) * (t)->srow + (int64_t)(j) * (t)->scol])
#define ZB(t, i, j) ((t)->z[(int64_t)(i) * (t)->srow + (int64_t)(j) * (t)->scol])

/* ---- worker threads over a range of rows --------------------------------
 * A job is a function applied to rows [lo, hi).  With T threads, thread i
 * (the caller is thread 0) takes rows [R*i/T, R*(i+1)/T) of the R rows, and
 * the caller returns once every share is done. */
typedef void (*orc_rows_fn)(orc_tab *t, void *arg, int64_t lo, int64_t hi);

struct orc_pool {
  int32_t threads;
  pthread_t *tid;
  pthread_mutex_t mu;
  pthread_cond_t cv;
  atomic_uint_fast64_t gen; /* bumped once per job */
  atomic_int done;          /* workers finished with the current job */
  int quit;
  orc_rows_fn fn;
  orc_tab *t;
  void *arg;
  int64_t nrows;
};

typedef struct { orc_pool *p; int32_t index; } orc_worker_arg;

static void share_of(int64_t nrows, int32_t threads, int32_t i, int64_t *lo, int64_t *hi) {
  *lo = nrows * i / threads;
  *hi = nrows * (i + 1) / threads;
}

static void *orc_worker(void *varg) {
  orc_worker_arg *wa = (orc_worker_arg *)varg;
  orc_pool *p = wa->p;
  int32_t index = wa->index;
  free(wa);
  uint_fast64_t seen = 0;
  for (;;) {
    uint_fast64_t g;
    long spins = 0;
    /* spin briefly (jobs come back to back inside a run), then sleep */
    while ((g = atomic_load_explicit(&p->gen, memory_order_acquire)) == seen) {
      if (++spins < (1L << 16)) continue;
      if (spins < (1L << 18)) { sched_yield(); continue; }
      pthread_mutex_lock(&p->mu);
      while ((g = atomic_load_explicit(&p->gen, memory_order_acquire)) == seen)
        pthread_cond_wait(&p->cv, &p->mu);
      pthread_mutex_unlock(&p->mu);
      break;
    }
    seen = g;
    if (p->quit) return NULL;
    int64_t lo, hi;
    share_of(p->nrows, p->threads, index, &lo, &hi);
    if (lo < hi) p->fn(p->t, p->arg, lo, hi);
    atomic_fetch_add_explicit(&p->done, 1, memory_order_acq_rel);
  }
}

static void pool_stop(orc_pool *p, int32_t started) {
  pthread_mutex_lock(&p->mu);
  p->quit = 1;
  atomic_fetch_add_explicit(&p->gen, 1, memory_order_release);
  pthread_cond_broadcast(&p->cv);
  pthread_mutex_unlock(&p->mu);
  for (int32_t i = 0; i < started; i++) pthread_join(p->tid[i], NULL);
  pthread_cond_destroy(&p->cv);
  pthread_mutex_destroy(&p->mu);
  free(p->tid);
  free(p);
}

/* Run fn over rows [0, nrows) on the tableau's threads. */
static void for_rows(orc_tab *t, orc_rows_fn fn, void *arg, int64_t nrows) {
  orc_pool *p = t->pool;
  if (!p) {
    fn(t, arg, 0, nrows);
    return;
  }
  p->fn = fn;
  p->t = t;
  p->arg = arg;
  p->nrows = nrows;
  atomic_store_explicit(&p->done, 0, memory_order_relaxed);
  pthread_mutex_lock(&p->mu);
  atomic_fetch_add_explicit(&p->gen, 1, memory_order_release);
  pthread_cond_broadcast(&p->cv);
  pthread_mutex_unlock(&p->mu);
  int64_t lo, hi;
  share_of(nrows, p->threads, 0, &lo, &hi);
  if (lo < hi) fn(t, arg, lo, hi);
  long spins = 0;
  while (atomic_load_explicit(&p->done, memory_order_acquire) != p->threads - 1)
    if (++spins > (1L << 18)) sched_yield();
}

/* Use `threads` threads (>= 1) for this tableau's row loops. */
int32_t orc_set_threads(orc_tab *t, int32_t threads) {
  if (threads < 1) return ORC_EINVAL;
  if (t->pool) {
    pool_stop(t->pool, t->pool->threads - 1);
    t->pool = NULL;
  }
  if (threads == 1) return ORC_OK;
  orc_pool *p = (orc_pool *)calloc(1, sizeof(orc_pool));
  if (!p) return ORC_ENOMEM;
  p->threads = threads;
  p->tid = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
  if (!p->tid) { free(p); return ORC_ENOMEM; }
  pthread_mutex_init(&p->mu, NULL);
  pthread_cond_init(&p->cv, NULL);
  atomic_init(&p->gen, 0);
  atomic_init(&p->done, 0);
  for (int32_t i = 1; i < threads; i++) {
    orc_worker_arg *wa = (orc_worker_arg *)malloc(sizeof(orc_worker_arg));
    if (wa) {
      wa->p = p;
      wa->index = i;
    }
    if (!wa || pthread_create(&p->tid[i - 1], NULL, orc_worker, wa) != 0) {
      free(wa);
      pool_stop(p, i - 1);
      return ORC_ENOMEM;
    }
  }
  t->pool = p;
  return ORC_OK;
}

int32_t orc_threads(const orc_tab *t) { return t->pool ? t->pool->threads : 1; }

/* ---- storage order ------------------------------------------------------ */

typedef struct { const uint8_t *src; uint8_t *dst; int64_t ss_row, ss_col; } reorder_job;

/* rows [lo, hi) of one array copied into the other order */
static void reorder_rows(orc_tab *t, void *arg, int64_t lo, int64_t hi) {
  const reorder_job *job = (const reorder_job *)arg;
  const int64_t n = t->n;
  for (int64_t i0 = lo; i0 < hi; i0 += 64) {
    const int64_t i1 = i0 + 64 < hi ? i0 + 64 : hi;
    for (int64_t j0 = 0; j0 < n; j0 += 64) {
      const int64_t j1 = j0 + 64 < n ? j0 + 64 : n;
      for (int64_t i = i0; i < i1; i++)
        for (int64_t j = j0; j < j1; j++)
          job->dst[i * t->srow + j * t->scol] = job->src[i * job->ss_row + j * job->ss_col];
    }
  }
}

/* Keep x and z row-major (rows = 1) or qubit-major (rows = 0). */
static void storage_order(orc_tab *t, int rows) {
  if (rows) t->row_gates = 0;
  if ((t->scol == 1) == (rows != 0)) return;
  const int64_t old_row = t->srow, old_col = t->scol;
  t->srow = rows ? t->n : 1;
  t->scol = rows ? 1 : t->rows;
  uint8_t **arr[2] = {&t->x, &t->z};
  for (int k = 0; k < 2; k++) {
    reorder_job job = {*arr[k], t->spare, old_row, old_col};
    for_rows(t, reorder_rows, &job, t->rows);
    t->spare = *arr[k];
    *arr[k] = job.dst;
  }
}

void orc_reset(orc_tab *t) {
  int64_t cells = (int64_t)t->n * t->rows;
  memset(t->x, 0, (size_t)cells);
  memset(t->z, 0, (size_t)cells);
  memset(t->r, 0, (size_t)t->rows);
  t->noise_counter = 0;
  /* |0^n>: destabilizer i = X_i, stabilizer n+i = Z_i, all signs + */
  for (int32_t i = 0; i < t->n; i++) {
    XB(t, i, i) = 1;
    ZB(t, t->n + i, i) = 1;
  }
}

orc_tab *orc_new(int32_t n) {
  if (n < 1) return NULL;
  orc_tab *t = (orc_tab *)calloc(1, sizeof(orc_tab));
  if (!t) return NULL;
  t->n = n;
  t->rows = 2 * (int64_t)n + 1;
  t->srow = 1;
  t->scol = t->rows;
  int64_t cells = (int64_t)n * t->rows;
  t->x = (uint8_t *)malloc((size_t)cells);
  t->z = (uint8_t *)malloc((size_t)cells);
  t->spare = (uint8_t *)malloc((size_t)cells);
  t->r = (uint8_t *)malloc((size_t)t->rows);
  if (!t->x || !t->z || !t->spare || !t->r) {
    free(t->x); free(t->z); free(t->spare); free(t->r); free(t);
    return NULL;
  }
  orc_reset(t);
  return t;
}

void orc_free(orc_tab *t) {
  if (!t) return;
  if (t->pool) pool_stop(t->pool, t->pool->threads - 1);
  free(t->x); free(t->z); free(t->spare); free(t->r); free(t);
}

int32_t orc_n(const orc_tab *t) { return t->n; }

/* before a gate rule: qubit-major order, unless few rules have run since the
 * last measurement */
static void gate_order(orc_tab *t) {
  if (t->scol == 1 && ++t->row_gates <= t->n / 16 + 16) return;
  storage_order(t, 0);
}

/* ---- AG's three gate rules, for every row i in [0, 2n) ----------------
 * Each rule is written for a range of rows; the public function runs it over
 * all 2n rows (split over the tableau's threads, if it has any). */

static void cnot_rows(orc_tab *t, void *arg, int64_t lo, int64_t hi) {
  const int32_t a = ((const int32_t *)arg)[0], b = ((const int32_t *)arg)[1];
  for (int64_t i = lo; i < hi; i++) {
    uint8_t xa = XB(t, i, a), za = ZB(t, i, a), xb = XB(t, i, b), zb = ZB(t, i, b);
    t->r[i] ^= (uint8_t)(xa & zb & (xb ^ za ^ 1));
    XB(t, i, b) = (uint8_t)(xb ^ xa);
    ZB(t, i, a) = (uint8_t)(za ^ zb);
  }
}

static void h_rows(orc_tab *t, void *arg, int64_t lo, int64_t hi) {
  const int32_t a = *(const int32_t *)arg;
  for (int64_t i = lo; i < hi; i++) {
    uint8_t xa = XB(t, i, a), za = ZB(t, i, a);
    t->r[i] ^= (uint8_t)(xa & za);
    XB(t, i, a) = za;
    ZB(t, i, a) = xa;
  }
}

static void s_rows(orc_tab *t, void *arg, int64_t lo, int64_t hi) {
  const int32_t a = *(const int32_t *)arg;
  for (int64_t i = lo; i < hi; i++) {
    uint8_t xa = XB(t, i, a), za = ZB(t, i, a);
    t->r[i] ^= (uint8_t)(xa & za);
    ZB(t, i, a) = (uint8_t)(za ^ xa);
  }
}

void orc_cnot(orc_tab *t, int32_t a, int32_t b) {
  int32_t ab[2] = {a, b};
  gate_order(t);
  for_rows(t, cnot_rows, ab, 2 * (int64_t)t->n);
}

void orc_h(orc_tab *t, int32_t a) {
  gate_order(t);
  for_rows(t, h_rows, &a, 2 * (int64_t)t->n);
}

void orc_s(orc_tab *t, int32_t a) {
  gate_order(t);
  for_rows(t, s_rows, &a, 2 * (int64_t)t->n);
}

/* ---- gates built from the three rules --------------------------------- */

void orc_z(orc_tab *t, int32_t a) { orc_s(t, a); orc_s(t, a); }
void orc_x(orc_tab *t, int32_t a) { orc_h(t, a); orc_z(t, a); orc_h(t, a); }
void orc_y(orc_tab *t, int32_t a) { orc_z(t, a); orc_x(t, a); }
void orc_sdg(orc_tab *t, int32_t a) { orc_s(t, a); orc_s(t, a); orc_s(t, a); }
void orc_cz(orc_tab *t, int32_t a, int32_t b) { orc_h(t, b); orc_cnot(t, a, b); orc_h(t, b); }
void orc_swap(orc_tab *t, int32_t a, int32_t b) {
  orc_cnot(t, a, b); orc_cnot(t, b, a); orc_cnot(t, a, b);
}

/* ---- rowsum ------------------------------------------------------------ */

/* AG's g: the power of i in P(x1,z1) * P(x2,z2). */
int32_t orc_g(int32_t x1, int32_t z1, int32_t x2, int32_t z2) {
  if (x1 == 0 && z1 == 0) return 0;
  if (x1 == 1 && z1 == 1) return z2 - x2;
  if (x1 == 1 && z1 == 0) return z2 * (2 * x2 - 1);
  return x2 * (1 - 2 * z2); /* x1 == 0, z1 == 1 */
}

/* AG rowsum(h, i): row h := row i * row h.  Returns ORC_EPHASE (and leaves
 * row h unchanged) when the exponent is odd, i.e. the rows anticommute. */
int32_t orc_rowsum(orc_tab *t, int64_t h, int64_t i) {
  /* g over its 16 arguments, indexed by x1 z1 x2 z2 (high to low bit) */
  int8_t g[16];
  for (int32_t k = 0; k < 16; k++)
    g[k] = (int8_t)orc_g((k >> 3) & 1, (k >> 2) & 1, (k >> 1) & 1, k & 1);
  const int64_t sc = t->scol;
  const uint8_t *xi = &XB(t, i, 0), *zi = &ZB(t, i, 0);
  uint8_t *xh = &XB(t, h, 0), *zh = &ZB(t, h, 0);
  int64_t sum = 2 * (int64_t)t->r[h] + 2 * (int64_t)t->r[i];
  for (int64_t j = 0; j < t->n; j++)
    sum += g[(xi[j * sc] << 3) | (zi[j * sc] << 2) | (xh[j * sc] << 1) | zh[j * sc]];
  int64_t m = ((sum % 4) + 4) % 4;
  if (m != 0 && m != 2) return ORC_EPHASE;
  t->r[h] = (uint8_t)(m == 2);
  for (int64_t j = 0; j < t->n; j++) {
    xh[j * sc] ^= xi[j * sc];
    zh[j * sc] ^= zi[j * sc];
  }
  return ORC_OK;
}

/* ---- Philox4x32-10 ----------------------------------------------------- */

static void philox_round(uint32_t c[4], const uint32_t k[2]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  uint64_t p0 = (uint64_t)M0 * c[0];
  uint64_t p1 = (uint64_t)M1 * c[2];
  uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  uint32_t n0 = hi1 ^ c[1] ^ k[0];
  uint32_t n2 = hi0 ^ c[3] ^ k[1];
  c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int round = 0; round < 10; round++) {
    if (round > 0) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }
    philox_round(c, k);
  }
  memcpy(out, c, sizeof c);
}

/* outcome bit of measurement index k of (circuit_id, shot) under seed */
int32_t orc_outcome_bit(uint64_t seed, uint64_t circuit_id, uint32_t shot, uint64_t k) {
  uint32_t ctr[4] = {(uint32_t)k, shot, (uint32_t)circuit_id, (uint32_t)(circuit_id >> 32)};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  return (int32_t)(out[0] & 1u);
}

/* ---- measurement (AG Sec. III) ----------------------------------------- */

/* Case 1's rowsums: every row i != p, p-n with x_ia = 1 takes rowsum(i, p).
 * Each writes only row i and reads row p, which none of them writes. */
typedef struct {
  int64_t p;
  int32_t a;
  atomic_int rc; /* the first error seen by any share */
} random_case_job;

static void random_case_rows(orc_tab *t, void *arg, int64_t lo, int64_t hi) {
  random_case_job *job = (random_case_job *)arg;
  const int64_t p = job->p, n = t->n;
  for (int64_t i = lo; i < hi; i++) {
    if (i == p || i == p - n || !XB(t, i, job->a)) continue;
    int32_t rc = orc_rowsum(t, i, p);
    if (rc != ORC_OK) {
      int expected = ORC_OK;
      atomic_compare_exchange_strong(&job->rc, &expected, rc);
      return;
    }
  }
}

/* Measure Z_a with the pre-drawn bit `rbit` for the random case.  Returns the
 * outcome (0/1) or a negative error; *deterministic is set to 1 or 0. */
int32_t orc_measure(orc_tab *t, int32_t a, int32_t rbit, int32_t *deterministic) {
  if (a < 0 || a >= t->n) return ORC_ERANGE;
  storage_order(t, 1);
  const int64_t n = t->n;
  int64_t p = -1;
  for (int64_t i = n; i < 2 * n; i++)
    if (XB(t, i, a)) { p = i; break; }
  if (p >= 0) {
    /* case 1: random outcome */
    random_case_job job = {p, a, ORC_OK};
    for_rows(t, random_case_rows, &job, 2 * n);
    if (job.rc != ORC_OK) return job.rc;
    for (int32_t j = 0; j < t->n; j++) {
      XB(t, p - n, j) = XB(t, p, j);
      ZB(t, p - n, j) = ZB(t, p, j);
      XB(t, p, j) = 0;
      ZB(t, p, j) = 0;
    }
    t->r[p - n] = t->r[p];
    ZB(t, p, a) = 1;
    t->r[p] = (uint8_t)(rbit & 1);
    if (deterministic) *deterministic = 0;
    return rbit & 1;
  }
  /* case 2: deterministic outcome, via the scratch row 2n */
  const int64_t s = 2 * n;
  for (int32_t j = 0; j < t->n; j++) { XB(t, s, j) = 0; ZB(t, s, j) = 0; }
  t->r[s] = 0;
  for (int64_t i = 0; i < n; i++) {
    if (!XB(t, i, a)) continue;
    int32_t rc = orc_rowsum(t, s, i + n);
    if (rc != ORC_OK) return rc;
  }
  if (deterministic) *deterministic = 1;
  return t->r[s];
}

/* ---- gate-list driver ---------------------------------------------------
 * Gate word: bits 63..56 op, 55..28 q1, 27..0 q2 (the library's format).
 * Ops: 0 I, 1 X, 2 Y, 3 Z, 4 H, 5 S, 6 SDG, 7 CNOT, 8 CZ, 9 SWAP, 10 MZ,
 * 11 MZR, 12 BARRIER.  Outcomes are appended to out[] (one byte each,
 * program order); det[] (optional) gets 1 for deterministic outcomes.
 * *meas_counter is the next measurement index and is advanced.  Returns the
 * number of outcomes written, or a negative error. */
int64_t orc_run(orc_tab *t, const uint64_t *gates, int64_t count, uint64_t seed,
                uint64_t circuit_id, uint32_t shot, uint64_t *meas_counter,
                uint8_t *out, int64_t out_cap, uint8_t *det) {
  int64_t nout = 0;
  for (int64_t gi = 0; gi < count; gi++) {
    uint64_t g = gates[gi];
    int32_t op = (int32_t)(g >> 56);
    int64_t q1 = (int64_t)((g >> 28) & 0xFFFFFFFull);
    int64_t q2 = (int64_t)(g & 0xFFFFFFFull);
    int two = (op == 7 || op == 8 || op == 9);
    if (op < 0 || op > 17) return ORC_EINVAL;
    if (op != 12 && q1 >= t->n) return ORC_ERANGE;
    if (two && (q2 >= t->n)) return ORC_ERANGE;
    if (two && q1 == q2) return ORC_EINVAL;
    int32_t a = (int32_t)q1, b = (int32_t)q2;
    switch (op) {
      case 0: case 12: break;
      case 1: orc_x(t, a); break;
      case 2: orc_y(t, a); break;
      case 3: orc_z(t, a); break;
      case 4: orc_h(t, a); break;
      case 5: orc_s(t, a); break;
      case 6: orc_sdg(t, a); break;
      case 7: orc_cnot(t, a, b); break;
      case 8: orc_cz(t, a, b); break;
      case 9: orc_swap(t, a, b); break;
      case 10: case 11: case 13: case 14: {
        /* MX, MY: rotate the measured Pauli onto Z_a, measure, rotate back */
        if (op == 14) orc_sdg(t, a);
        if (op == 13 || op == 14) orc_h(t, a);
        uint64_t k = (*meas_counter)++;
        int32_t rbit = orc_outcome_bit(seed, circuit_id, shot, k);
        int32_t d = 0;
        int32_t m = orc_measure(t, a, rbit, &d);
        if (m < 0) return m;
        if (nout >= out_cap) return ORC_EINVAL;
        out[nout] = (uint8_t)m;
        if (det) det[nout] = (uint8_t)d;
        nout++;
        if (op == 11 && m == 1) orc_x(t, a);
        if (op == 13 || op == 14) orc_h(t, a);
        if (op == 14) orc_s(t, a);
        break;
      }
      case 15: case 16: case 17: {
        uint64_t j = t->noise_counter++;
        uint32_t ctr[4] = {(uint32_t)j, shot, (uint32_t)circuit_id, (uint32_t)(circuit_id >> 32)};
        uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ 0x4E4F4953u};
        uint32_t w[4];
        orc_philox4x32_10(ctr, key, w);
        if ((w[0] >> 4) < (uint32_t)q2) {
          uint32_t which = op == 16 ? 0u : op == 17 ? 2u : (uint32_t)(((uint64_t)w[1] * 3u) >> 32);
          if (which == 0) orc_x(t, a);
          else if (which == 1) orc_y(t, a);
          else orc_z(t, a);
        }
        break;
      }
      default: return ORC_EINVAL;
    }
  }
  return nout;
}

/* ---- expectation value of a Pauli string ------------------------------ */

/* <psi|P|psi> for the Pauli with codes p[0..n) (0 I, 1 X, 2 Z, 3 Y; bit 0 is
 * x, bit 1 is z).  AG Sec. III: the state is the +1 eigenstate of the
 * stabilizer rows, so <P> = 0 when P anticommutes with one of them; otherwise
 * +-P is the product of the stabilizer rows n+i over the destabilizers i that
 * anticommute with P (the product the deterministic measurement forms for
 * Z_a), built here in the scratch row by rowsum, and <P> is its sign.
 * Returns -1, 0 or +1; ORC_EINVAL for a bad code; ORC_EPHASE if the product
 * is not +-P.  Rows 0..2n-1 are unchanged. */
int32_t orc_expect(orc_tab *t, const uint8_t *p) {
  int32_t n = t->n;
  int64_t s = 2 * (int64_t)n;
  for (int32_t j = 0; j < n; j++)
    if (p[j] > 3) return ORC_EINVAL;
  storage_order(t, 1);
  uint8_t *anti = (uint8_t *)calloc((size_t)t->rows, 1);
  if (!anti) return ORC_ENOMEM;
  for (int64_t i = 0; i < 2 * (int64_t)n; i++) {
    int c = 0;
    for (int32_t j = 0; j < n; j++)
      c ^= (XB(t, i, j) & (p[j] >> 1)) ^ (ZB(t, i, j) & (p[j] & 1));
    anti[i] = (uint8_t)c;
  }
  for (int64_t i = n; i < 2 * (int64_t)n; i++)
    if (anti[i]) { free(anti); return 0; }
  for (int32_t j = 0; j < n; j++) { XB(t, s, j) = 0; ZB(t, s, j) = 0; }
  t->r[s] = 0;
  for (int64_t i = 0; i < n; i++) {
    if (!anti[i]) continue;
    int32_t rc = orc_rowsum(t, s, n + i);
    if (rc < 0) { free(anti); return rc; }
  }
  free(anti);
  for (int32_t j = 0; j < n; j++)
    if (XB(t, s, j) != (p[j] & 1) || ZB(t, s, j) != (p[j] >> 1)) return ORC_EPHASE;
  return t->r[s] ? -1 : 1;
}

/* ---- import / export: row-major unpacked bits, rows 0..2n-1 ------------ */

void orc_get(const orc_tab *t, uint8_t *x, uint8_t *z, uint8_t *r) {
  int64_t n = t->n;
  for (int64_t i = 0; i < 2 * n; i++) {
    for (int64_t j = 0; j < n; j++) {
      x[i * n + j] = XB(t, i, j);
      z[i * n + j] = ZB(t, i, j);
    }
    r[i] = t->r[i];
  }
}

void orc_set(orc_tab *t, const uint8_t *x, const uint8_t *z, const uint8_t *r) {
  int64_t n = t->n;
  for (int64_t i = 0; i < 2 * n; i++) {
    for (int64_t j = 0; j < n; j++) {
      XB(t, i, j) = x[i * n + j] & 1;
      ZB(t, i, j) = z[i * n + j] & 1;
    }
    t->r[i] = r[i] & 1;
  }
}
