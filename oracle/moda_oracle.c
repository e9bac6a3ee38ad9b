/*
 * Plain CPU oracle for the multi-objective Digital Annealer (MDA) of
 * "Multi-objective QUBO Solver: Bi-objective Quadratic Assignment Problem"
 * (Ayodele et al., arXiv 2205.13399).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file.  The CUDA library shares no
 * code, header, helper or table generator with it; neither includes the
 * other.
 *
 * It computes, step by step and in the paper's order, with explicit QUBO
 * matrices (the GPU path never stores Q):
 *   - Sec. 2.2, Eq. cqap / Sec. 2.3 Eq. bf: the cost QUBO of objective k in
 *     the upper-triangular form printed in the worked example
 *     (C_pp = Q_pp, C_pq = Q_pq + Q_qp for p < q,
 *      Q_(i,u),(j,v) = h_ij * d_uv, bit p = i*n + u = facility i at
 *      location u, as the worked example encodes it);
 *   - Sec. 2.2, Eq. gqap: the constraint QUBO G and its constant p_g,
 *     obtained by expanding each squared row / column term;
 *   - Sec. 3.2, Eq. vermap / wvermaa: the penalty weight w (alpha = w / 2),
 *     with the row sums taken over the symmetric P = C + C^T (the bound on
 *     the change of one flip, which is what the text says w is);
 *   - Sec. 3.3, Eq. wqubom: Y = R + alpha_1 G and Z = S + alpha_2 G.  G has
 *     only even entries and p_g = 2n, so alpha * G is integral for any
 *     integer w and every energy is an exact int64;
 *   - Sec. 3.1, Eq. cale: Delta E_i = (1 - 2 x_i)(P_ii + sum_{j!=i} P_ij x_j),
 *     P = Q + Q^T with P_ii = Q_ii (the printed equation carries a stray
 *     factor x_i; E(y) = E(x) + Delta E_i, stated beside it, fixes this form);
 *   - Sec. 3.3, Alg. 3 (MDA) with the strict (Eq. pacceptms) or lenient
 *     (Eq. pacceptml) acceptance rule and the explorative (Alg. 4) or
 *     exploitative (Alg. 5) archive update; the escape either jumps to a
 *     random archive member (Alg. 3) or raises the DA's energy offset by
 *     beta (Alg. 1, Eq. paccepts).
 *
 * Random draws come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 * "Parallel Random Numbers: As Easy as 1, 2, 3", SC'11), keyed by the seed
 * and addressed by (bit group, step, replica, purpose), written here from
 * that paper's definition.  The acceptance variate of a bit is the top 16
 * bits of its Philox word, u = (idx + 0.5) / 65536, and the test is
 * "accept iff (double)a <= delta * (-ln u)", the strict product of
 * exp(-max(0, dE_k)/delta) being exp(-(sum_k max(0, dE_k))/delta) and the
 * lenient maximum being exp(-min_k max(0, dE_k)/delta).
 *
 * Compile with -ffp-contract=off: the only floating point on the path is
 * the cooling product and one multiply per acceptance test, both plain
 * IEEE double operations.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10                                                             */
/* ------------------------------------------------------------------------ */

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                          uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Purposes of a draw (the fourth counter word). */
enum { TAG_ACCEPT = 0, TAG_SELECT = 1, TAG_RESTART = 2, TAG_EXPLOIT = 3,
       TAG_INIT = 4 };

static uint32_t draw_word(uint64_t seed, uint32_t group, uint32_t step,
                          uint32_t replica, uint32_t tag, int word) {
  uint32_t ctr[4] = {group, step, replica, tag};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  oracle_philox4x32_10(ctr, key, out);
  return out[word];
}

/* Uniform choice of one of `count` items from a 32-bit word: floor(u*count
 * / 2^32). */
static int64_t pick(uint32_t u, int64_t count) {
  return (int64_t)(((uint64_t)u * (uint64_t)count) >> 32);
}

/* ------------------------------------------------------------------------ */
/* Temperature schedule and the -ln(u) table                                 */
/* ------------------------------------------------------------------------ */

/* delta used at iterations 1..count of Alg. 3: before each iteration's
 * Delta E, "if delta > delta_f then delta <- delta * (1 - xi)". */
void oracle_schedule(double delta0, double deltaf, double xi, int64_t count,
                     double *out) {
  double delta = delta0;
  double factor = 1.0 - xi;
  for (int64_t t = 0; t < count; ++t) {
    if (delta > deltaf) delta = delta * factor;
    out[t] = delta;
  }
}

/* T[idx] = -ln((idx + 0.5) / 65536), idx = top 16 bits of a Philox word. */
void oracle_neglog_table(double *T) {
  for (int idx = 0; idx < 65536; ++idx)
    T[idx] = -log(((double)idx + 0.5) / 65536.0);
}

/* ------------------------------------------------------------------------ */
/* QUBO construction                                                         */
/* ------------------------------------------------------------------------ */

/* Upper-triangular cost QUBO of Eq. cqap for flows H and distances D
 * (n x n, row-major).  C is m x m, m = n*n. */
void oracle_cost_qubo(int n, const int64_t *H, const int64_t *D, int64_t *C) {
  int64_t m = (int64_t)n * n;
  memset(C, 0, sizeof(int64_t) * (size_t)(m * m));
  for (int i = 0; i < n; ++i)
    for (int u = 0; u < n; ++u)
      for (int j = 0; j < n; ++j)
        for (int v = 0; v < n; ++v) {
          int64_t p = (int64_t)i * n + u, q = (int64_t)j * n + v;
          int64_t qpq = H[i * n + j] * D[u * n + v];
          if (p <= q)
            C[p * m + q] += qpq;
          else
            C[q * m + p] += qpq;
        }
}

/* Upper-triangular constraint QUBO of Eq. gqap and its constant p_g.  Each
 * squared term (1 - sum_{p in S} x_p)^2, S a row or a column of the n x n
 * assignment matrix, expands (x_p^2 = x_p) to
 *   1 - sum_{p in S} x_p + 2 * sum_{p<q in S} x_p x_q. */
void oracle_constraint_qubo(int n, int64_t *G, int64_t *pg) {
  int64_t m = (int64_t)n * n;
  memset(G, 0, sizeof(int64_t) * (size_t)(m * m));
  int64_t constant = 0;
  int64_t *members = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  for (int rowcol = 0; rowcol < 2; ++rowcol)
    for (int g = 0; g < n; ++g) {
      for (int k = 0; k < n; ++k)
        members[k] = rowcol == 0 ? (int64_t)g * n + k : (int64_t)k * n + g;
      constant += 1;
      for (int k = 0; k < n; ++k) G[members[k] * m + members[k]] -= 1;
      for (int k = 0; k < n; ++k)
        for (int l = k + 1; l < n; ++l) {
          int64_t p = members[k], q = members[l];
          if (p > q) { int64_t s = p; p = q; q = s; }
          G[p * m + q] += 2;
        }
    }
  free(members);
  *pg = constant;
}

/* Eq. vermap on the symmetric P = C + C^T (P_ii = C_ii): the largest change
 * of x^T C x that one flip can make. */
int64_t oracle_penalty_w(int64_t m, const int64_t *C) {
  int64_t w = INT64_MIN;
  for (int64_t i = 0; i < m; ++i) {
    int64_t neg = -C[i * m + i], pos = C[i * m + i];
    for (int64_t j = 0; j < m; ++j) {
      if (j == i) continue;
      int64_t pij = C[i * m + j] + C[j * m + i];
      if (pij < 0) neg -= pij;
      if (pij > 0) pos += pij;
    }
    if (neg > w) w = neg;
    if (pos > w) w = pos;
  }
  return w;
}

/* x^T U x for an upper-triangular U. */
int64_t oracle_quadratic(int64_t m, const int64_t *U, const uint8_t *x) {
  int64_t e = 0;
  for (int64_t p = 0; p < m; ++p) {
    if (!x[p]) continue;
    for (int64_t q = p; q < m; ++q)
      if (x[q]) e += U[p * m + q];
  }
  return e;
}

/* ------------------------------------------------------------------------ */
/* Instance: Y, Z (Eq. wqubom) and their symmetric P matrices (Eq. cale)     */
/* ------------------------------------------------------------------------ */

typedef struct oracle_instance {
  int n;
  int64_t m;
  int64_t w[2];        /* penalty weight w_k, alpha_k = w_k / 2 */
  int64_t offset[2];   /* constant term alpha_k * p_g of E_k */
  int64_t *C[2];       /* upper-triangular cost QUBOs R, S */
  int64_t *G;          /* upper-triangular constraint QUBO */
  int64_t pg;
  int64_t *Y[2];       /* upper-triangular Y, Z */
  int64_t *P[2];       /* symmetric P of Y, Z (diagonal = Y_pp) */
} oracle_instance;

void oracle_instance_free(oracle_instance *inst) {
  if (!inst) return;
  for (int k = 0; k < 2; ++k) {
    free(inst->C[k]);
    free(inst->Y[k]);
    free(inst->P[k]);
  }
  free(inst->G);
  free(inst);
}

/* penalty_kind 0: w_k from Eq. vermap on the objective's own cost QUBO
 * (Sec. 3.3); 1: the caller's w1, w2. */
oracle_instance *oracle_instance_new(int n, const int64_t *F1,
                                     const int64_t *F2, const int64_t *D,
                                     int penalty_kind, int64_t w1,
                                     int64_t w2) {
  if (n < 1) return NULL;
  oracle_instance *inst = (oracle_instance *)calloc(1, sizeof(*inst));
  if (!inst) return NULL;
  int64_t m = (int64_t)n * n;
  size_t bytes = sizeof(int64_t) * (size_t)(m * m);
  inst->n = n;
  inst->m = m;
  inst->G = (int64_t *)malloc(bytes);
  for (int k = 0; k < 2; ++k) {
    inst->C[k] = (int64_t *)malloc(bytes);
    inst->Y[k] = (int64_t *)malloc(bytes);
    inst->P[k] = (int64_t *)malloc(bytes);
    if (!inst->C[k] || !inst->Y[k] || !inst->P[k]) {
      oracle_instance_free(inst);
      return NULL;
    }
  }
  if (!inst->G) {
    oracle_instance_free(inst);
    return NULL;
  }
  oracle_cost_qubo(n, F1, D, inst->C[0]);
  oracle_cost_qubo(n, F2, D, inst->C[1]);
  oracle_constraint_qubo(n, inst->G, &inst->pg);
  for (int k = 0; k < 2; ++k) {
    inst->w[k] = penalty_kind == 0 ? oracle_penalty_w(m, inst->C[k])
                                   : (k == 0 ? w1 : w2);
    /* alpha_k * G with alpha_k = w_k / 2 and every G entry even. */
    for (int64_t e = 0; e < m * m; ++e)
      inst->Y[k][e] = inst->C[k][e] + inst->w[k] * (inst->G[e] / 2);
    inst->offset[k] = inst->w[k] * (inst->pg / 2);
    for (int64_t p = 0; p < m; ++p)
      for (int64_t q = 0; q < m; ++q)
        inst->P[k][p * m + q] =
            p == q ? inst->Y[k][p * m + p]
                   : inst->Y[k][p * m + q] + inst->Y[k][q * m + p];
  }
  return inst;
}

int64_t oracle_instance_w(const oracle_instance *inst, int k) {
  return inst->w[k];
}
int64_t oracle_instance_m(const oracle_instance *inst) { return inst->m; }

void oracle_instance_copy(const oracle_instance *inst, int which, int64_t *out) {
  /* which: 0 = R, 1 = S, 2 = G, 3 = Y, 4 = Z */
  const int64_t *src = which == 0   ? inst->C[0]
                       : which == 1 ? inst->C[1]
                       : which == 2 ? inst->G
                       : which == 3 ? inst->Y[0]
                                    : inst->Y[1];
  memcpy(out, src, sizeof(int64_t) * (size_t)(inst->m * inst->m));
}

int64_t oracle_instance_pg(const oracle_instance *inst) { return inst->pg; }

/* E_k(x) = x^T Y_k x + alpha_k p_g (Eq. mqap / wqubom). */
int64_t oracle_energy(const oracle_instance *inst, int k, const uint8_t *x) {
  return oracle_quadratic(inst->m, inst->Y[k], x) + inst->offset[k];
}
/* c_k(x) = x^T C_k x (Eq. bf). */
int64_t oracle_cost(const oracle_instance *inst, int k, const uint8_t *x) {
  return oracle_quadratic(inst->m, inst->C[k], x);
}
/* g(x) = x^T G x + p_g (Eq. gqap). */
int64_t oracle_constraint(const oracle_instance *inst, const uint8_t *x) {
  return oracle_quadratic(inst->m, inst->G, x) + inst->pg;
}

/* ------------------------------------------------------------------------ */
/* MDA (Alg. 3)                                                              */
/* ------------------------------------------------------------------------ */

typedef struct oracle_params {
  int64_t I_max;
  double delta0, deltaf, xi;
  int64_t beta;       /* energy-offset increase (escape = 1 only) */
  int64_t archive_size; /* s */
  int accept;         /* 0 strict (Eq. pacceptms), 1 lenient (Eq. pacceptml) */
  int archive;        /* 0 explorative (Alg. 4), 1 exploitative (Alg. 5) */
  int escape;         /* 0 jump to an archive member (Alg. 3),
                         1 raise the energy offset by beta (Alg. 1) */
  int check;          /* 1: recompute energies and fields from scratch
                         every iteration and fail on any mismatch */
  uint64_t seed;
  int normalize;      /* 1: Sec. 4.2 normalisation, see oracle_norm_scale */
  int64_t snap_every; /* > 0: copy the archive after every iteration t with
                         t % snap_every == 0 (the per-iteration archive
                         behind Fig. mdasl's hypervolume trace) */
} oracle_params;

/* Sec. 4.2: "the largest QUBO coefficient representing any objective QUBO
 * R and S" is set to 2^23.  Objective k is scaled by
 *   s_k = 2^23 / max_{p <= q} C_k[p][q]      (1 if that maximum is 0)
 * over its upper-triangular cost QUBO as the worked example prints it.
 * Y_k = s_k R_k + alpha'_k G with alpha'_k from s_k R_k is s_k times the
 * unscaled Y_k, so E'_k = s_k E_k; dominance between states is unchanged
 * and only the acceptance test (Eqs. pacceptms / pacceptml / paccepts)
 * sees the scale.  The scaled quantities are doubles, evaluated in IEEE
 * double as written, operation by operation. */
double oracle_norm_scale(const oracle_instance *inst, int k) {
  const int64_t m = inst->m;
  int64_t mx = 0;
  for (int64_t p = 0; p < m; ++p)
    for (int64_t q = p; q < m; ++q)
      if (inst->C[k][p * m + q] > mx) mx = inst->C[k][p * m + q];
  return mx > 0 ? 8388608.0 / (double)mx : 1.0;
}

/* Per-replica outputs. */
typedef struct oracle_result {
  int64_t archive_count;
  int64_t *archive_E;    /* [s][2] */
  uint8_t *archive_bits; /* [s][m] */
  uint8_t *x_final;      /* [m] */
  int64_t E_final[2];
  int64_t stats[4];      /* flips, jumps to the archive, escapes with an empty
                            archive, offset raises */
  int64_t *trace;        /* [I_max][3] E1, E2, event, or NULL */
  int64_t *snap_count;   /* [I_max / snap_every] archive sizes, or NULL */
  int64_t *snap_E;       /* [I_max / snap_every][s][2] */
  uint8_t *snap_bits;    /* [I_max / snap_every][s][m] */
} oracle_result;

/* x dominates y (Sec. 3.3): no worse in both energies and not equivalent. */
static int dominates(int64_t x1, int64_t x2, int64_t y1, int64_t y2) {
  return x1 <= y1 && x2 <= y2 && !(x1 == y1 && x2 == y2);
}

static void archive_store(oracle_result *res, int64_t slot, int64_t m,
                          const uint8_t *x, const int64_t E[2]) {
  res->archive_E[slot * 2 + 0] = E[0];
  res->archive_E[slot * 2 + 1] = E[1];
  memcpy(res->archive_bits + slot * m, x, (size_t)m);
}

/* Alg. 4: replace the first archive member that x dominates, otherwise add
 * x when the archive is not full. */
static void update_explorative(oracle_result *res, int64_t s, int64_t m,
                               const uint8_t *x, const int64_t E[2]) {
  for (int64_t y = 0; y < res->archive_count; ++y) {
    if (dominates(E[0], E[1], res->archive_E[2 * y], res->archive_E[2 * y + 1])) {
      archive_store(res, y, m, x, E);
      return;
    }
  }
  if (res->archive_count < s) {
    archive_store(res, res->archive_count, m, x, E);
    res->archive_count += 1;
  }
}

/* Alg. 5: if no archive member dominates x, replace a random member of
 * B = {y : x dominates y}, or add x when B is empty and the archive is not
 * full.  The random member is B[floor(u |B| / 2^32)], B in slot order, u
 * being the exploit draw of this iteration. */
static void update_exploitative(oracle_result *res, int64_t s, int64_t m,
                                const uint8_t *x, const int64_t E[2],
                                int64_t *Bbuf, uint32_t u) {
  int64_t nb = 0;
  int dominated = 0;
  for (int64_t y = 0; y < res->archive_count; ++y) {
    int64_t y1 = res->archive_E[2 * y], y2 = res->archive_E[2 * y + 1];
    if (dominates(E[0], E[1], y1, y2)) Bbuf[nb++] = y;
    if (dominates(y1, y2, E[0], E[1])) dominated = 1;
  }
  if (dominated) return;
  if (nb > 0) {
    archive_store(res, Bbuf[pick(u, nb)], m, x, E);
  } else if (res->archive_count < s) {
    archive_store(res, res->archive_count, m, x, E);
    res->archive_count += 1;
  }
}

/* One archive update on energies alone (no bits), for replaying hand-made
 * sequences: kind 0 explorative, 1 exploitative with draw u. */
int oracle_archive_update(int kind, int64_t s, int64_t *count, int64_t *E,
                          const int64_t Enew[2], uint32_t u) {
  oracle_result res;
  memset(&res, 0, sizeof(res));
  res.archive_count = *count;
  res.archive_E = E;
  uint8_t dummy = 0;
  res.archive_bits = &dummy;
  int64_t *Bbuf = (int64_t *)malloc(sizeof(int64_t) * (size_t)(s + 1));
  if (!Bbuf) return -2;
  if (kind == 0)
    update_explorative(&res, s, 0, &dummy, Enew);
  else
    update_exploitative(&res, s, 0, &dummy, Enew, Bbuf, u);
  free(Bbuf);
  *count = res.archive_count;
  return 0;
}

/* Acceptance of one bit with penalty a at temperature delta for the draws
 * of counters (g, step, replica, 0), g = 0..groups-1, word 0..3: returns
 * how many of the 4 * groups tests accept. */
int64_t oracle_accept_count(int64_t a, double delta, uint64_t seed,
                            uint32_t step, uint32_t replica, int64_t groups) {
  double T[1];
  int64_t acc = 0;
  for (int64_t g = 0; g < groups; ++g) {
    uint32_t ctr[4] = {(uint32_t)g, step, replica, TAG_ACCEPT};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    for (int w = 0; w < 4; ++w) {
      T[0] = -log(((double)(out[w] >> 16) + 0.5) / 65536.0);
      if ((double)a <= delta * T[0]) acc++;
    }
  }
  return acc;
}

/* phi_k[p] = sum_{q != p} P_k[p][q] x_q */
static void fields_from_scratch(const oracle_instance *inst, const uint8_t *x,
                                int64_t *phi0, int64_t *phi1) {
  int64_t m = inst->m;
  for (int64_t p = 0; p < m; ++p) {
    phi0[p] = 0;
    phi1[p] = 0;
  }
  for (int64_t q = 0; q < m; ++q) {
    if (!x[q]) continue;
    const int64_t *r0 = inst->P[0] + q * m, *r1 = inst->P[1] + q * m;
    for (int64_t p = 0; p < m; ++p) {
      if (p == q) continue;
      phi0[p] += r0[p];
      phi1[p] += r1[p];
    }
  }
}

/* Runs Alg. 3 for one replica.  Returns 0, or a negative code: -1 bad
 * arguments, -2 out of memory, -3 a check (params.check) failed. */
int oracle_mda_run(const oracle_instance *inst, const oracle_params *prm,
                   uint32_t replica, oracle_result *res) {
  const int64_t m = inst->m;
  const int64_t s = prm->archive_size > 0 ? prm->archive_size : m;
  if (prm->I_max < 0 || prm->I_max > 0xFFFFFFFFll) return -1;
  int rc = 0;
  uint8_t *x = (uint8_t *)calloc((size_t)m, 1);
  int64_t *phi0 = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
  int64_t *phi1 = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
  int64_t *dE0 = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
  int64_t *dE1 = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
  int64_t *accepted = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
  int64_t *Bbuf = (int64_t *)malloc(sizeof(int64_t) * (size_t)(s + 1));
  int64_t *chk0 = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
  int64_t *chk1 = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
  double *T = (double *)malloc(sizeof(double) * 65536);
  if (!x || !phi0 || !phi1 || !dE0 || !dE1 || !accepted || !Bbuf || !chk0 ||
      !chk1 || !T) {
    rc = -2;
    goto done;
  }
  oracle_neglog_table(T);
  memset(res->stats, 0, sizeof(res->stats));
  res->archive_count = 0;

  /* "x <- a random binary solution": bit k is bit (k mod 32) of word
   * (k / 32) mod 4 of the draw for group k / 128 at step 0. */
  for (int64_t k = 0; k < m; ++k) {
    uint32_t w = draw_word(prm->seed, (uint32_t)(k >> 7), 0, replica,
                           TAG_INIT, (int)((k >> 5) & 3));
    x[k] = (uint8_t)((w >> (k & 31)) & 1u);
  }
  int64_t E[2] = {oracle_energy(inst, 0, x), oracle_energy(inst, 1, x)};
  fields_from_scratch(inst, x, phi0, phi1);

  double delta = prm->delta0;
  const double factor = 1.0 - prm->xi;
  int64_t Eoff = 0;
  const double sc0 = prm->normalize ? oracle_norm_scale(inst, 0) : 1.0;
  const double sc1 = prm->normalize ? oracle_norm_scale(inst, 1) : 1.0;

  for (int64_t it = 1; it <= prm->I_max; ++it) {
    const uint32_t step = (uint32_t)it;
    if (delta > prm->deltaf) delta = delta * factor;

    /* Eq. cale for both objectives. */
    for (int64_t p = 0; p < m; ++p) {
      int64_t sgn = 1 - 2 * (int64_t)x[p];
      dE0[p] = sgn * (inst->P[0][p * m + p] + phi0[p]);
      dE1[p] = sgn * (inst->P[1][p * m + p] + phi1[p]);
    }

    /* Parallel trial: every bit is tested. */
    int64_t count = 0;
    for (int64_t p = 0; p < m; ++p) {
      uint32_t w = draw_word(prm->seed, (uint32_t)(p >> 2), step, replica,
                             TAG_ACCEPT, (int)(p & 3));
      double t = T[w >> 16];
      if (!prm->normalize) {
        int64_t e0 = dE0[p], e1 = dE1[p];
        if (prm->escape == 1) {
          e0 -= Eoff;
          e1 -= Eoff;
        }
        int64_t a0 = e0 > 0 ? e0 : 0, a1 = e1 > 0 ? e1 : 0;
        int64_t a = prm->accept == 0 ? a0 + a1 : (a0 < a1 ? a0 : a1);
        if ((double)a <= delta * t) accepted[count++] = p;
      } else {
        /* normalised: s_k Delta E_k - E_offset per objective, in doubles */
        double e0 = sc0 * (double)dE0[p], e1 = sc1 * (double)dE1[p];
        if (prm->escape == 1) {
          e0 = e0 - (double)Eoff;
          e1 = e1 - (double)Eoff;
        }
        double a0 = e0 > 0 ? e0 : 0.0, a1 = e1 > 0 ? e1 : 0.0;
        double a = prm->accept == 0 ? a0 + a1 : (a0 < a1 ? a0 : a1);
        if (a <= delta * t) accepted[count++] = p;
      }
    }

    int64_t event;
    if (count > 0) {
      /* Choose one recorded flip at random: rank floor(u c / 2^32) in
       * ascending bit order. */
      uint32_t u = draw_word(prm->seed, 0, step, replica, TAG_SELECT, 0);
      int64_t q = accepted[pick(u, count)];
      int64_t sgn = x[q] ? -1 : 1; /* +1 when the bit turns on */
      E[0] += dE0[q];
      E[1] += dE1[q];
      x[q] ^= 1;
      const int64_t *r0 = inst->P[0] + q * m, *r1 = inst->P[1] + q * m;
      for (int64_t p = 0; p < m; ++p) {
        if (p == q) continue;
        phi0[p] += sgn * r0[p];
        phi1[p] += sgn * r1[p];
      }
      Eoff = 0;
      if (prm->archive == 0)
        update_explorative(res, s, m, x, E);
      else
        update_exploitative(
            res, s, m, x, E, Bbuf,
            draw_word(prm->seed, 0, step, replica, TAG_EXPLOIT, 0));
      res->stats[0] += 1;
      event = q;
    } else if (prm->escape == 0) {
      if (res->archive_count > 0) {
        uint32_t u = draw_word(prm->seed, 0, step, replica, TAG_RESTART, 0);
        int64_t slot = pick(u, res->archive_count);
        memcpy(x, res->archive_bits + slot * m, (size_t)m);
        E[0] = res->archive_E[2 * slot];
        E[1] = res->archive_E[2 * slot + 1];
        fields_from_scratch(inst, x, phi0, phi1);
        res->stats[1] += 1;
        event = -1 - slot;
      } else {
        res->stats[2] += 1;
        event = INT64_MIN;
      }
    } else {
      Eoff += prm->beta;
      res->stats[3] += 1;
      event = INT64_MIN;
    }
    if (res->snap_count && prm->snap_every > 0 && it % prm->snap_every == 0) {
      const int64_t j = it / prm->snap_every - 1;
      res->snap_count[j] = res->archive_count;
      memcpy(res->snap_E + j * s * 2, res->archive_E, sizeof(int64_t) * (size_t)(2 * s));
      memcpy(res->snap_bits + j * s * m, res->archive_bits, (size_t)(s * m));
    }
    if (res->trace) {
      res->trace[(it - 1) * 3 + 0] = E[0];
      res->trace[(it - 1) * 3 + 1] = E[1];
      res->trace[(it - 1) * 3 + 2] = event;
    }
    if (prm->check) {
      if (E[0] != oracle_energy(inst, 0, x) ||
          E[1] != oracle_energy(inst, 1, x)) {
        rc = -3;
        goto done;
      }
      fields_from_scratch(inst, x, chk0, chk1);
      for (int64_t p = 0; p < m; ++p)
        if (chk0[p] != phi0[p] || chk1[p] != phi1[p]) {
          rc = -3;
          goto done;
        }
    }
  }
  memcpy(res->x_final, x, (size_t)m);
  res->E_final[0] = E[0];
  res->E_final[1] = E[1];

done:
  free(x); free(phi0); free(phi1); free(dE0); free(dE1); free(accepted);
  free(Bbuf); free(chk0); free(chk1); free(T);
  return rc;
}

/* Flat-array entry point for ctypes.  Outputs per replica r:
 *   count[r], E[r][s][2], bits[r][s][m], x_final[r][m], E_final[r][2],
 *   stats[r][4], trace[r][I_max][3] (trace may be NULL). */
typedef struct {
  const oracle_instance *inst;
  const oracle_params *prm;
  const uint32_t *replicas;
  int64_t n_rep;
  int64_t *count, *E, *E_final, *stats, *trace;
  uint8_t *bits, *x_final;
  int64_t *snap_count, *snap_E;
  uint8_t *snap_bits;
  int64_t next;
  int rc;
  pthread_mutex_t lock;
} batch_job;

static void *batch_worker(void *arg) {
  batch_job *job = (batch_job *)arg;
  const int64_t m = job->inst->m;
  const int64_t s = job->prm->archive_size > 0 ? job->prm->archive_size : m;
  for (;;) {
    pthread_mutex_lock(&job->lock);
    int64_t r = job->next++;
    pthread_mutex_unlock(&job->lock);
    if (r >= job->n_rep) break;
    oracle_result res;
    res.archive_E = job->E + r * s * 2;
    res.archive_bits = job->bits + r * s * m;
    res.x_final = job->x_final + r * m;
    res.trace = job->trace ? job->trace + r * job->prm->I_max * 3 : NULL;
    const int64_t ns = job->prm->snap_every > 0 ? job->prm->I_max / job->prm->snap_every : 0;
    res.snap_count = job->snap_count && ns > 0 ? job->snap_count + r * ns : NULL;
    res.snap_E = job->snap_E ? job->snap_E + r * ns * s * 2 : NULL;
    res.snap_bits = job->snap_bits ? job->snap_bits + r * ns * s * m : NULL;
    int rc = oracle_mda_run(job->inst, job->prm, job->replicas[r], &res);
    job->count[r] = res.archive_count;
    job->E_final[r * 2 + 0] = res.E_final[0];
    job->E_final[r * 2 + 1] = res.E_final[1];
    memcpy(job->stats + r * 4, res.stats, sizeof(res.stats));
    if (rc != 0) {
      pthread_mutex_lock(&job->lock);
      job->rc = rc;
      pthread_mutex_unlock(&job->lock);
    }
  }
  return NULL;
}

int oracle_mda_run_many(const oracle_instance *inst, const oracle_params *prm,
                        int64_t n_rep, const uint32_t *replicas, int nthreads,
                        int64_t *count, int64_t *E, uint8_t *bits,
                        uint8_t *x_final, int64_t *E_final, int64_t *stats,
                        int64_t *trace, int64_t *snap_count, int64_t *snap_E,
                        uint8_t *snap_bits) {
  batch_job job;
  memset(&job, 0, sizeof(job));
  job.snap_count = snap_count;
  job.snap_E = snap_E;
  job.snap_bits = snap_bits;
  job.inst = inst; job.prm = prm; job.replicas = replicas; job.n_rep = n_rep;
  job.count = count; job.E = E; job.bits = bits; job.x_final = x_final;
  job.E_final = E_final; job.stats = stats; job.trace = trace;
  pthread_mutex_init(&job.lock, NULL);
  if (nthreads < 1) nthreads = 1;
  if (nthreads > n_rep) nthreads = (int)(n_rep > 0 ? n_rep : 1);
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
  int started = 0;
  for (int i = 0; i < nthreads; ++i)
    if (pthread_create(&th[i], NULL, batch_worker, &job) == 0) started++;
  if (started == 0) batch_worker(&job);
  for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
  free(th);
  pthread_mutex_destroy(&job.lock);
  return job.rc;
}

/* ------------------------------------------------------------------------ */
/* SB-DA (Sec. 3.2, Alg. 2) and the DA it calls (Sec. 3.1, Alg. 1)          */
/* ------------------------------------------------------------------------ */

/* The scalarised QUBO of Alg. 2 for the weight gamma = gnum / gden, kept
 * integral by scaling everything by gden (temperatures and the offset rate
 * are scaled by the same factor, which leaves exp(-a / delta) unchanged):
 *   C = gnum R + (gden - gnum) S                      (Alg. 2, cost line)
 *   alpha = w / 2, w by Eq. vermap on C               (Alg. 2, alpha line)
 *   Q = C + alpha G                                   (G entries are even) */
typedef struct oracle_squbo {
  int n;
  int64_t m;
  int64_t w;
  int64_t cmax;    /* largest coefficient of C, p <= q (Sec. 4.2) */
  int64_t offset;  /* alpha p_g */
  int64_t *Q;      /* upper triangular */
  int64_t *P;      /* symmetric, diagonal = Q_pp (Eq. cale) */
} oracle_squbo;

void oracle_squbo_free(oracle_squbo *q) {
  if (!q) return;
  free(q->Q);
  free(q->P);
  free(q);
}

oracle_squbo *oracle_sbda_qubo(const oracle_instance *inst, int64_t gnum,
                               int64_t gden) {
  if (gden < 1 || gnum < 0 || gnum > gden) return NULL;
  const int64_t m = inst->m;
  oracle_squbo *q = (oracle_squbo *)calloc(1, sizeof(*q));
  if (!q) return NULL;
  q->n = inst->n;
  q->m = m;
  q->Q = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m * m));
  q->P = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m * m));
  int64_t *C = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m * m));
  if (!q->Q || !q->P || !C) {
    free(C);
    oracle_squbo_free(q);
    return NULL;
  }
  for (int64_t e = 0; e < m * m; ++e)
    C[e] = gnum * inst->C[0][e] + (gden - gnum) * inst->C[1][e];
  q->cmax = 0;
  for (int64_t p = 0; p < m; ++p)
    for (int64_t r = p; r < m; ++r)
      if (C[p * m + r] > q->cmax) q->cmax = C[p * m + r];
  q->w = oracle_penalty_w(m, C);
  for (int64_t e = 0; e < m * m; ++e) q->Q[e] = C[e] + q->w * (inst->G[e] / 2);
  q->offset = q->w * (inst->pg / 2);
  for (int64_t p = 0; p < m; ++p)
    for (int64_t r = 0; r < m; ++r)
      q->P[p * m + r] = p == r ? q->Q[p * m + p] : q->Q[p * m + r] + q->Q[r * m + p];
  free(C);
  return q;
}

int64_t oracle_squbo_w(const oracle_squbo *q) { return q->w; }

/* Sec. 4.2 for the scalarised QUBO: s = 2^23 / (largest coefficient of its
 * cost part C), 1 if that is 0.  The gden factor of C cancels in s C. */
double oracle_squbo_scale(const oracle_squbo *q) {
  return q->cmax > 0 ? 8388608.0 / (double)q->cmax : 1.0;
}

/* E(x) = x^T Q x + alpha p_g */
int64_t oracle_squbo_energy(const oracle_squbo *q, const uint8_t *x) {
  return oracle_quadratic(q->m, q->Q, x) + q->offset;
}

typedef struct oracle_da_params {
  int64_t I_max;
  double delta0, deltaf, xi;  /* scaled by gden unless normalize */
  int64_t beta;               /* scaled by gden unless normalize */
  uint64_t seed;
  int normalize;              /* 1: the acceptance test sees s Delta E - E_off
                                 in IEEE double (s = oracle_squbo_scale), the
                                 temperatures and the offset in the units of
                                 the normalised QUBO */
} oracle_da_params;

/* Alg. 1 for one replica with the draws of Alg. 3 (same Philox counters).
 * "Best solution found": the lowest energy among the states reached by
 * accepted flips, the earliest on ties; the initial state when no flip is
 * ever accepted.  stats: [flips, offset raises]. */
int oracle_da_run(const oracle_squbo *q, const oracle_da_params *prm,
                  uint32_t replica, uint8_t *best_x, int64_t *best_E,
                  uint8_t *x_final, int64_t *E_final, int64_t *stats) {
  const int64_t m = q->m;
  if (prm->I_max < 0 || prm->I_max > 0xFFFFFFFFll) return -1;
  int rc = 0;
  uint8_t *x = (uint8_t *)calloc((size_t)m, 1);
  int64_t *phi = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
  int64_t *dE = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
  int64_t *accepted = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
  double *T = (double *)malloc(sizeof(double) * 65536);
  if (!x || !phi || !dE || !accepted || !T) {
    rc = -2;
    goto done;
  }
  oracle_neglog_table(T);
  stats[0] = stats[1] = 0;
  /* "x <- a random binary solution" (the init draws of Alg. 3) */
  for (int64_t k = 0; k < m; ++k) {
    uint32_t w = draw_word(prm->seed, (uint32_t)(k >> 7), 0, replica, TAG_INIT,
                           (int)((k >> 5) & 3));
    x[k] = (uint8_t)((w >> (k & 31)) & 1u);
  }
  int64_t E = oracle_squbo_energy(q, x);
  for (int64_t p = 0; p < m; ++p) phi[p] = 0;
  for (int64_t r = 0; r < m; ++r) {
    if (!x[r]) continue;
    for (int64_t p = 0; p < m; ++p)
      if (p != r) phi[p] += q->P[r * m + p];
  }
  memcpy(best_x, x, (size_t)m);
  *best_E = E;
  int have_best = 0;
  double delta = prm->delta0;
  const double factor = 1.0 - prm->xi;
  const double scale = oracle_squbo_scale(q);
  int64_t Eoff = 0;
  for (int64_t it = 1; it <= prm->I_max; ++it) {
    const uint32_t step = (uint32_t)it;
    if (delta > prm->deltaf) delta = delta * factor;
    /* calculate Delta E (Eq. cale) */
    for (int64_t p = 0; p < m; ++p)
      dE[p] = (1 - 2 * (int64_t)x[p]) * (q->P[p * m + p] + phi[p]);
    /* propose every flip with Delta E_i - E_offset (Eq. paccepts) */
    int64_t count = 0;
    for (int64_t p = 0; p < m; ++p) {
      uint32_t w = draw_word(prm->seed, (uint32_t)(p >> 2), step, replica, TAG_ACCEPT,
                             (int)(p & 3));
      if (!prm->normalize) {
        int64_t e = dE[p] - Eoff;
        int64_t a = e > 0 ? e : 0;
        if ((double)a <= delta * T[w >> 16]) accepted[count++] = p;
      } else {
        /* normalised QUBO: s Delta E_i - E_offset, in doubles */
        double e = scale * (double)dE[p];
        e = e - (double)Eoff;
        double a = e > 0 ? e : 0.0;
        if (a <= delta * T[w >> 16]) accepted[count++] = p;
      }
    }
    if (count > 0) {
      uint32_t u = draw_word(prm->seed, 0, step, replica, TAG_SELECT, 0);
      int64_t r = accepted[pick(u, count)];
      int64_t sgn = x[r] ? -1 : 1;
      E += dE[r];
      x[r] ^= 1;
      for (int64_t p = 0; p < m; ++p)
        if (p != r) phi[p] += sgn * q->P[r * m + p];
      Eoff = 0;
      stats[0] += 1;
      if (!have_best || E < *best_E) {
        memcpy(best_x, x, (size_t)m);
        *best_E = E;
        have_best = 1;
      }
    } else {
      Eoff += prm->beta;
      stats[1] += 1;
    }
  }
  memcpy(x_final, x, (size_t)m);
  *E_final = E;
done:
  free(x); free(phi); free(dE); free(accepted); free(T);
  return rc;
}

typedef struct {
  const oracle_squbo *q;
  const oracle_da_params *prm;
  const uint32_t *replicas;
  int64_t n_rep;
  uint8_t *best_x, *x_final;
  int64_t *best_E, *E_final, *stats;
  int64_t next;
  int rc;
  pthread_mutex_t lock;
} da_job;

static void *da_worker(void *arg) {
  da_job *job = (da_job *)arg;
  const int64_t m = job->q->m;
  for (;;) {
    pthread_mutex_lock(&job->lock);
    int64_t r = job->next++;
    pthread_mutex_unlock(&job->lock);
    if (r >= job->n_rep) break;
    int rc = oracle_da_run(job->q, job->prm, job->replicas[r], job->best_x + r * m,
                           job->best_E + r, job->x_final + r * m, job->E_final + r,
                           job->stats + 2 * r);
    if (rc != 0) {
      pthread_mutex_lock(&job->lock);
      job->rc = rc;
      pthread_mutex_unlock(&job->lock);
    }
  }
  return NULL;
}

int oracle_da_run_many(const oracle_squbo *q, const oracle_da_params *prm, int64_t n_rep,
                       const uint32_t *replicas, int nthreads, uint8_t *best_x,
                       int64_t *best_E, uint8_t *x_final, int64_t *E_final,
                       int64_t *stats) {
  da_job job;
  memset(&job, 0, sizeof(job));
  job.q = q; job.prm = prm; job.replicas = replicas; job.n_rep = n_rep;
  job.best_x = best_x; job.best_E = best_E; job.x_final = x_final;
  job.E_final = E_final; job.stats = stats;
  pthread_mutex_init(&job.lock, NULL);
  if (nthreads < 1) nthreads = 1;
  if (nthreads > n_rep) nthreads = (int)(n_rep > 0 ? n_rep : 1);
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
  int started = 0;
  for (int i = 0; i < nthreads; ++i)
    if (pthread_create(&th[i], NULL, da_worker, &job) == 0) started++;
  if (started == 0) da_worker(&job);
  for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
  free(th);
  pthread_mutex_destroy(&job.lock);
  return job.rc;
}

/* ------------------------------------------------------------------------ */
/* Explicit QUBOs with K objectives (Alg. 3 on stored matrices)             */
/* ------------------------------------------------------------------------ */

/* K objectives, each an explicit upper-triangular QUBO Q_k of m bits
 * (E_k(x) = x^T Q_k x), with P_k = Q_k + Q_k^T off the diagonal and
 * P_pp = Q_pp (Eq. cale).  Nothing about the QAP is assumed: any penalty
 * is part of Q_k. */
typedef struct oracle_kqubo {
  int K;
  int64_t m;
  int64_t *Q;  /* [K][m][m] */
  int64_t *P;  /* [K][m][m] */
} oracle_kqubo;

void oracle_kqubo_free(oracle_kqubo *q) {
  if (!q) return;
  free(q->Q);
  free(q->P);
  free(q);
}

oracle_kqubo *oracle_kqubo_new(int K, int64_t m, const int64_t *Q) {
  if (K < 1 || K > 8 || m < 1) return NULL;
  oracle_kqubo *q = (oracle_kqubo *)calloc(1, sizeof(*q));
  if (!q) return NULL;
  const size_t mm = (size_t)(m * m);
  q->K = K;
  q->m = m;
  q->Q = (int64_t *)malloc(sizeof(int64_t) * mm * (size_t)K);
  q->P = (int64_t *)malloc(sizeof(int64_t) * mm * (size_t)K);
  if (!q->Q || !q->P) {
    oracle_kqubo_free(q);
    return NULL;
  }
  for (int k = 0; k < K; ++k) {
    const int64_t *Qk = Q + (size_t)k * mm;
    int64_t *Uk = q->Q + (size_t)k * mm, *Pk = q->P + (size_t)k * mm;
    for (int64_t p = 0; p < m; ++p)
      for (int64_t r = 0; r < m; ++r) Uk[p * m + r] = r >= p ? Qk[p * m + r] : 0;
    for (int64_t p = 0; p < m; ++p)
      for (int64_t r = 0; r < m; ++r)
        Pk[p * m + r] = p == r ? Uk[p * m + p] : Uk[p * m + r] + Uk[r * m + p];
  }
  return q;
}

int64_t oracle_kqubo_energy(const oracle_kqubo *q, int k, const uint8_t *x) {
  return oracle_quadratic(q->m, q->Q + (size_t)k * (size_t)(q->m * q->m), x);
}

static int dominates_k(int K, const int64_t *a, const int64_t *b) {
  int strict = 0;
  for (int k = 0; k < K; ++k) {
    if (a[k] > b[k]) return 0;
    if (a[k] < b[k]) strict = 1;
  }
  return strict;
}

/* Alg. 3 for one replica on K objectives, with Alg. 3's Philox counters;
 * archive energies [s][K], trace [I_max][K + 1] (energies, event).  The
 * strict rule sums max(0, Delta E_k) over the objectives, the lenient one
 * takes their minimum (Eqs. pacceptms / pacceptml with K factors).  Returns
 * 0, -1 bad arguments, -2 out of memory, -3 a check failed. */
int oracle_kqubo_run(const oracle_kqubo *q, const oracle_params *prm, uint32_t replica,
                     int64_t *count, int64_t *arch_E, uint8_t *arch_bits, uint8_t *x_final,
                     int64_t *E_final, int64_t *stats, int64_t *trace) {
  const int K = q->K;
  const int64_t m = q->m;
  const size_t mm = (size_t)(m * m);
  const int64_t s = prm->archive_size > 0 ? prm->archive_size : m;
  if (prm->I_max < 0 || prm->I_max > 0xFFFFFFFFll) return -1;
  int rc = 0;
  uint8_t *x = (uint8_t *)calloc((size_t)m, 1);
  int64_t *phi = (int64_t *)calloc((size_t)(K * m), sizeof(int64_t));
  int64_t *dE = (int64_t *)malloc(sizeof(int64_t) * (size_t)(K * m));
  int64_t *accepted = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
  int64_t *Bbuf = (int64_t *)malloc(sizeof(int64_t) * (size_t)(s + 1));
  double *T = (double *)malloc(sizeof(double) * 65536);
  int64_t E[8];
  if (!x || !phi || !dE || !accepted || !Bbuf || !T) {
    rc = -2;
    goto done;
  }
  oracle_neglog_table(T);
  for (int j = 0; j < 4; ++j) stats[j] = 0;
  *count = 0;
  for (int64_t p = 0; p < m; ++p) {
    uint32_t w = draw_word(prm->seed, (uint32_t)(p >> 7), 0, replica, TAG_INIT,
                           (int)((p >> 5) & 3));
    x[p] = (uint8_t)((w >> (p & 31)) & 1u);
  }
#define KQ_FIELDS()                                                        \
  do {                                                                     \
    for (int64_t e = 0; e < K * m; ++e) phi[e] = 0;                        \
    for (int64_t r = 0; r < m; ++r) {                                      \
      if (!x[r]) continue;                                                 \
      for (int k = 0; k < K; ++k) {                                        \
        const int64_t *row = q->P + (size_t)k * mm + (size_t)r * (size_t)m; \
        for (int64_t p = 0; p < m; ++p)                                    \
          if (p != r) phi[k * m + p] += row[p];                            \
      }                                                                    \
    }                                                                      \
  } while (0)
  KQ_FIELDS();
  for (int k = 0; k < K; ++k) E[k] = oracle_kqubo_energy(q, k, x);
  double delta = prm->delta0;
  const double factor = 1.0 - prm->xi;
  int64_t Eoff = 0;
  for (int64_t it = 1; it <= prm->I_max; ++it) {
    const uint32_t step = (uint32_t)it;
    if (delta > prm->deltaf) delta = delta * factor;
    for (int k = 0; k < K; ++k)
      for (int64_t p = 0; p < m; ++p)
        dE[k * m + p] = (1 - 2 * (int64_t)x[p]) *
                        (q->P[(size_t)k * mm + (size_t)(p * m + p)] + phi[k * m + p]);
    int64_t cnt = 0;
    for (int64_t p = 0; p < m; ++p) {
      int64_t a = 0;
      for (int k = 0; k < K; ++k) {
        int64_t e = dE[k * m + p];
        if (prm->escape == 1) e -= Eoff;
        const int64_t ak = e > 0 ? e : 0;
        if (prm->accept == 0) a += ak;
        else a = (k == 0 || ak < a) ? ak : a;
      }
      uint32_t w = draw_word(prm->seed, (uint32_t)(p >> 2), step, replica, TAG_ACCEPT,
                             (int)(p & 3));
      if ((double)a <= delta * T[w >> 16]) accepted[cnt++] = p;
    }
    int64_t event = INT64_MIN;
    if (cnt > 0) {
      uint32_t u = draw_word(prm->seed, 0, step, replica, TAG_SELECT, 0);
      const int64_t r = accepted[pick(u, cnt)];
      const int64_t sgn = x[r] ? -1 : 1;
      for (int k = 0; k < K; ++k) E[k] += dE[k * m + r];
      x[r] ^= 1;
      for (int k = 0; k < K; ++k) {
        const int64_t *row = q->P + (size_t)k * mm + (size_t)r * (size_t)m;
        for (int64_t p = 0; p < m; ++p)
          if (p != r) phi[k * m + p] += sgn * row[p];
      }
      Eoff = 0;
      /* Alg. 4 / Alg. 5 with K-dimensional dominance */
      int64_t target = -1;
      if (prm->archive == 0) {
        for (int64_t y = 0; y < *count && target < 0; ++y)
          if (dominates_k(K, E, arch_E + y * K)) target = y;
        if (target < 0 && *count < s) target = (*count)++;
      } else {
        int64_t nb = 0;
        int dominated = 0;
        for (int64_t y = 0; y < *count; ++y) {
          if (dominates_k(K, E, arch_E + y * K)) Bbuf[nb++] = y;
          if (dominates_k(K, arch_E + y * K, E)) dominated = 1;
        }
        if (!dominated) {
          if (nb > 0)
            target = Bbuf[pick(draw_word(prm->seed, 0, step, replica, TAG_EXPLOIT, 0), nb)];
          else if (*count < s)
            target = (*count)++;
        }
      }
      if (target >= 0) {
        memcpy(arch_E + target * K, E, sizeof(int64_t) * (size_t)K);
        memcpy(arch_bits + target * m, x, (size_t)m);
      }
      stats[0] += 1;
      event = r;
    } else if (prm->escape == 0) {
      if (*count > 0) {
        uint32_t u = draw_word(prm->seed, 0, step, replica, TAG_RESTART, 0);
        const int64_t slot = pick(u, *count);
        memcpy(x, arch_bits + slot * m, (size_t)m);
        memcpy(E, arch_E + slot * K, sizeof(int64_t) * (size_t)K);
        KQ_FIELDS();
        stats[1] += 1;
        event = -1 - slot;
      } else {
        stats[2] += 1;
      }
    } else {
      Eoff += prm->beta;
      stats[3] += 1;
    }
    if (trace) {
      for (int k = 0; k < K; ++k) trace[(it - 1) * (K + 1) + k] = E[k];
      trace[(it - 1) * (K + 1) + K] = event;
    }
    if (prm->check)
      for (int k = 0; k < K; ++k)
        if (E[k] != oracle_kqubo_energy(q, k, x)) {
          rc = -3;
          goto done;
        }
  }
#undef KQ_FIELDS
  memcpy(x_final, x, (size_t)m);
  memcpy(E_final, E, sizeof(int64_t) * (size_t)K);
done:
  free(x); free(phi); free(dE); free(accepted); free(Bbuf); free(T);
  return rc;
}
