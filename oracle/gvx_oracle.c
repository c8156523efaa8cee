/*
 * gvx CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is the slow, obviously correct reference that the GPU library is checked against.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header, constant or helper with the CUDA library under
 * paper_2312_02756_gb300/csrc, and it never calls it.
 *
 * Two tiers:
 *   O1 ("definition", orc_*_def): each operation written out exactly as it is defined, evaluated
 *      in IEEE binary128 (long double on aarch64, __float128 + libquadmath on x86_64) and rounded
 *      to double once at the end.  binary128 is used because the plain definition
 *      m = sqrt(E^2 - |p|^2) loses up to log10(E^2/m^2) digits to cancellation; with 113 bits the
 *      rounding error stays far below the 1e-12 relative gate even at E^2/m^2 ~ 1e16.
 *   O2 ("fp64", orc_*_fp64): the same quantities from different, cancellation-free identities in
 *      plain double.  Fast enough to run over whole inputs on the host; it is also the timed CPU
 *      baseline.  O1 and O2 use different formulas, so their agreement pins both.
 *
 * Paper references (GenVectorX, arXiv 2312.02756):
 *   Sec. 4.1 and Fig. 1: InvariantMasses -- two arrays of Lorentz vectors given in any 4-D
 *     coordinate system; per index the two vectors are added and mass() of the sum is stored.
 *   Sec. 4.1: ApplyBoost -- a 4-D Lorentz transformation held as a 4x4 matrix and applied to every
 *     vector of an array.
 *   Sec. 3.1: vectors are templated on the coordinate system (here PtEtaPhiM in, PxPyPzE out).
 *   Sec. 6 (future work, RDataFrame analyses): per-event combinatorics -- the jagged form.
 * The paper prints no formula for the coordinate conversion or the boost matrix; the standard
 * relations used here (and their readings) are listed beside each function.
 *
 * Layouts: every 4-vector array is row-major n x 4 doubles.  PtEtaPhiM rows are (pt, eta, phi, m);
 * PxPyPzE rows are (px, py, pz, E).  Velocities are rows of 3 doubles (bx, by, bz).
 *
 * Parity pins: every function here is pinned by the CPU tests (closed forms, invariants, special
 * cases, finite differences, O1/O2 cross-agreement); none is "parity unpinned".
 */
#include <float.h>
#include <math.h>
#include <pthread.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>

#if LDBL_MANT_DIG == 113
typedef long double qreal;
#define Q_SIN sinl
#define Q_COS cosl
#define Q_SINH sinhl
#define Q_COSH coshl
#define Q_SQRT sqrtl
#define Q_BITS 113
#elif defined(__SIZEOF_FLOAT128__)
#include <quadmath.h>
typedef __float128 qreal;
#define Q_SIN sinq
#define Q_COS cosq
#define Q_SINH sinhq
#define Q_COSH coshq
#define Q_SQRT sqrtq
#define Q_BITS FLT128_MANT_DIG
#else
#error "the definition oracle needs IEEE binary128 arithmetic"
#endif

/* Mantissa bits of the extended type (113 for binary128); the tests assert it. */
int orc_precision_bits(void) { return Q_BITS; }

/* ------------------------------------------------------------------------------------------ */
/* A tiny thread fan-out: [0, n) is split into nthreads contiguous ranges.                     */

typedef void (*range_fn)(void *ctx, int64_t lo, int64_t hi);
typedef struct {
  range_fn fn;
  void *ctx;
  int64_t lo, hi;
} range_job;

static void *range_job_run(void *p) {
  range_job *j = (range_job *)p;
  j->fn(j->ctx, j->lo, j->hi);
  return NULL;
}

static void run_ranges(range_fn fn, void *ctx, int64_t n, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if (nthreads == 1 || n < 2 * nthreads) {
    fn(ctx, 0, n);
    return;
  }
  pthread_t tid[256];
  range_job job[256];
  int started[256];
  for (int t = 0; t < nthreads; t++) {
    job[t].fn = fn;
    job[t].ctx = ctx;
    job[t].lo = n * t / nthreads;
    job[t].hi = n * (t + 1) / nthreads;
    started[t] = pthread_create(&tid[t], NULL, range_job_run, &job[t]) == 0;
    if (!started[t]) range_job_run(&job[t]);
  }
  for (int t = 0; t < nthreads; t++)
    if (started[t]) pthread_join(tid[t], NULL);
}

/* ------------------------------------------------------------------------------------------ */
/* O1: definitions in binary128                                                               */

/* PtEtaPhiM -> PxPyPzE (Sec. 3.1 coordinate systems; the conversion that v1[id] + v2[id] in
 * Fig. 1 performs before adding):
 *   px = pt cos(phi), py = pt sin(phi), pz = pt sinh(eta), E = sqrt(px^2 + py^2 + pz^2 + m^2).
 * Reading: the stored m enters only through m^2 (its sign is ignored). */
static void leg_to_cartesian_q(const double *leg, qreal out[4]) {
  qreal pt = leg[0], eta = leg[1], phi = leg[2], m = leg[3];
  qreal px = pt * Q_COS(phi);
  qreal py = pt * Q_SIN(phi);
  qreal pz = pt * Q_SINH(eta);
  out[0] = px;
  out[1] = py;
  out[2] = pz;
  out[3] = Q_SQRT(px * px + py * py + pz * pz + m * m);
}

/* mass() of a PxPyPzE vector: sqrt(E^2 - |p|^2).  A negative E^2 - |p|^2 (possible only through
 * rounding here) returns -sqrt(-(E^2 - |p|^2)), GenVector's convention for spacelike vectors. */
static qreal lv_mass_q(const qreal v[4]) {
  qreal m2 = v[3] * v[3] - (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  return m2 >= 0 ? Q_SQRT(m2) : -Q_SQRT(-m2);
}

static double pair_mass_def(const double *a, const double *b) {
  qreal va[4], vb[4], w[4];
  leg_to_cartesian_q(a, va);
  leg_to_cartesian_q(b, vb);
  for (int k = 0; k < 4; k++) w[k] = va[k] + vb[k];
  return (double)lv_mass_q(w);
}

typedef struct {
  const double *a, *b;
  double *m;
} mass_ctx;

static void mass_def_range(void *p, int64_t lo, int64_t hi) {
  mass_ctx *c = (mass_ctx *)p;
  for (int64_t i = lo; i < hi; i++) c->m[i] = pair_mass_def(c->a + 4 * i, c->b + 4 * i);
}

/* Invariant mass of each pair (Sec. 4.1, Fig. 1): m[i] = mass(v1[i] + v2[i]). */
void orc_mass_def(const double *a, const double *b, int64_t n, double *m, int nthreads) {
  mass_ctx c = {a, b, m};
  run_ranges(mass_def_range, &c, n, nthreads);
}

/* The same definition evaluated in plain double: no tier uses it as a reference; the tests
 * report its error to show why O1 runs in binary128. */
void orc_mass_naive_fp64(const double *a, const double *b, int64_t n, double *m) {
  for (int64_t i = 0; i < n; i++) {
    double w[4] = {0, 0, 0, 0};
    const double *legs[2] = {a + 4 * i, b + 4 * i};
    for (int l = 0; l < 2; l++) {
      double pt = legs[l][0], eta = legs[l][1], phi = legs[l][2], mm = legs[l][3];
      double px = pt * cos(phi), py = pt * sin(phi), pz = pt * sinh(eta);
      w[0] += px;
      w[1] += py;
      w[2] += pz;
      w[3] += sqrt(px * px + py * py + pz * pz + mm * mm);
    }
    double m2 = w[3] * w[3] - (w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    m[i] = m2 >= 0 ? sqrt(m2) : -sqrt(-m2);
  }
}

/* Jacobian of one leg's PtEtaPhiM -> PxPyPzE conversion, J[r][c] = d v_r / d x_c with rows
 * (px, py, pz, E) and columns (pt, eta, phi, m), v = leg_to_cartesian_q(leg):
 *     px: ( cos phi,      0,           -pt sin phi, 0    )
 *     py: ( sin phi,      0,            pt cos phi, 0    )
 *     pz: ( sinh eta,     pt cosh eta,  0,          0    )
 *     E : ((px cos phi + py sin phi + pz sinh eta)/E, pz pt cosh eta / E,
 *          (-px pt sin phi + py pt cos phi)/E,  m/E )
 * Reading: a massless leg (m = 0) has E = pt cosh(eta), whose derivatives are used as they
 * stand, so that a leg at pt = 0, m = 0 gets the one-sided (pt >= 0) derivative and dE/dm = 0. */
static void leg_jacobian_q(const double *leg, const qreal v[4], qreal J[4][4]) {
  qreal pt = leg[0], eta = leg[1], phi = leg[2], mm = leg[3];
  qreal c = Q_COS(phi), s = Q_SIN(phi), sh = Q_SINH(eta), ch = Q_COSH(eta);
  qreal px = v[0], py = v[1], pz = v[2], e = v[3];
  qreal rows[4][4] = {
      {c, 0, -pt * s, 0},
      {s, 0, pt * c, 0},
      {sh, pt * ch, 0, 0},
      {0, 0, 0, 0},
  };
  for (int r = 0; r < 4; r++)
    for (int k = 0; k < 4; k++) J[r][k] = rows[r][k];
  if (mm == 0) {
    J[3][0] = ch;
    J[3][1] = pt * sh;
  } else {
    J[3][0] = (px * c + py * s + pz * sh) / e;
    J[3][1] = pz * pt * ch / e;
    J[3][2] = (-px * pt * s + py * pt * c) / e;
    J[3][3] = mm / e;
  }
}

/* dm/d(pt, eta, phi, m) of both legs of the pair mass, by the chain rule through the definition:
 * dm/d(Px,Py,Pz,E) of the summed vector = (-Px, -Py, -Pz, E) / m, times each leg's Jacobian.
 * Reading: where m <= 0 the gradient is zero (m is not differentiable at 0). */
static void pair_mass_dm_q(const double *a, const double *b, qreal ga[4], qreal gb[4]) {
  qreal v[2][4], w[4];
  leg_to_cartesian_q(a, v[0]);
  leg_to_cartesian_q(b, v[1]);
  for (int k = 0; k < 4; k++) w[k] = v[0][k] + v[1][k];
  qreal m = lv_mass_q(w);
  const double *legs[2] = {a, b};
  qreal *outs[2] = {ga, gb};
  if (!(m > 0)) {
    for (int l = 0; l < 2; l++)
      for (int k = 0; k < 4; k++) outs[l][k] = 0;
    return;
  }
  qreal dmdv[4] = {-w[0] / m, -w[1] / m, -w[2] / m, w[3] / m};
  for (int l = 0; l < 2; l++) {
    qreal J[4][4];
    leg_jacobian_q(legs[l], v[l], J);
    for (int k = 0; k < 4; k++) {
      qreal acc = 0;
      for (int r = 0; r < 4; r++) acc += dmdv[r] * J[r][k];
      outs[l][k] = acc;
    }
  }
}

/* Gradient of the pair mass times the upstream gradient gm, rounded once. */
static void pair_mass_grad_def(const double *a, const double *b, double gm, double *ga,
                               double *gb) {
  qreal qa[4], qb[4];
  pair_mass_dm_q(a, b, qa, qb);
  for (int k = 0; k < 4; k++) {
    ga[k] = (double)(qa[k] * (qreal)gm);
    gb[k] = (double)(qb[k] * (qreal)gm);
  }
}

typedef struct {
  const double *a, *b, *gm;
  double *ga, *gb;
} mass_grad_ctx;

static void mass_grad_def_range(void *p, int64_t lo, int64_t hi) {
  mass_grad_ctx *c = (mass_grad_ctx *)p;
  for (int64_t i = lo; i < hi; i++)
    pair_mass_grad_def(c->a + 4 * i, c->b + 4 * i, c->gm[i], c->ga + 4 * i, c->gb + 4 * i);
}

/* ga[i], gb[i] = gm[i] * d m[i] / d(pt, eta, phi, m) of leg a and leg b. */
void orc_mass_grad_def(const double *a, const double *b, const double *gm, int64_t n, double *ga,
                       double *gb, int nthreads) {
  mass_grad_ctx c = {a, b, gm, ga, gb};
  run_ranges(mass_grad_def_range, &c, n, nthreads);
}

/* The boost matrix (Sec. 4.1: ApplyBoost applies a 4x4 Lorentz matrix).  Index order is
 * (x, y, z, t) to match PxPyPzE.  For a velocity beta with b2 = |beta|^2 < 1:
 *   gamma = 1 / sqrt(1 - b2)
 *   L[t][t] = gamma,  L[i][t] = L[t][i] = gamma beta_i,
 *   L[i][j] = delta_ij + (gamma - 1) beta_i beta_j / b2.
 * Readings: "boost by +beta" (a vector at rest acquires velocity +beta); beta = 0 gives the
 * identity (the limit of the formula); |beta| >= 1 gives NaN everywhere. */
static int boost_matrix_q(const double *beta, qreal L[4][4]) {
  qreal bx = beta[0], by = beta[1], bz = beta[2];
  qreal b[3] = {bx, by, bz};
  qreal b2 = bx * bx + by * by + bz * bz;
  if (!(b2 < 1)) return 0;
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) L[i][j] = (i == j) ? 1 : 0;
  if (b2 == 0) return 1;
  qreal g = 1 / Q_SQRT(1 - b2);
  qreal c = (g - 1) / b2;
  for (int i = 0; i < 3; i++) {
    for (int j = 0; j < 3; j++) L[i][j] += c * b[i] * b[j];
    L[i][3] = g * b[i];
    L[3][i] = g * b[i];
  }
  L[3][3] = g;
  return 1;
}

/* Boost matrix rounded to double, row-major (x, y, z, t); NaN when |beta| >= 1. */
void orc_boost_matrix_def(const double *beta, double *L16) {
  qreal L[4][4];
  int ok = boost_matrix_q(beta, L);
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) L16[4 * i + j] = ok ? (double)L[i][j] : NAN;
}

typedef struct {
  const double *v, *beta;
  int64_t stride;
  double *out;
} boost_ctx;

static void boost_def_range(void *p, int64_t lo, int64_t hi) {
  boost_ctx *c = (boost_ctx *)p;
  for (int64_t i = lo; i < hi; i++) {
    qreal L[4][4];
    const double *vi = c->v + 4 * i;
    double *oi = c->out + 4 * i;
    if (!boost_matrix_q(c->beta + 3 * c->stride * i, L)) {
      for (int k = 0; k < 4; k++) oi[k] = NAN;
      continue;
    }
    for (int r = 0; r < 4; r++) {
      qreal acc = 0;
      for (int k = 0; k < 4; k++) acc += L[r][k] * (qreal)vi[k];
      oi[r] = (double)acc;
    }
  }
}

/* out[i] = L(beta[i * stride]) v[i]; stride 1 gives each vector its own velocity, stride 0
 * applies beta[0] to all (Sec. 4.1 ApplyBoost, one array of vectors). */
void orc_boost_def(const double *v, const double *beta, int64_t beta_stride, int64_t n,
                   double *out, int nthreads) {
  boost_ctx c = {v, beta, beta_stride, out};
  run_ranges(boost_def_range, &c, n, nthreads);
}

/* Gradient of the boost by the chain rule through the matrix definition.
 *   grad_v = L^T gout  (L is symmetric, so L gout).
 *   grad_beta_k = sum_ij gout_i (dL_ij / dbeta_k) v_j, with dgamma/dbeta_k = gamma^3 beta_k,
 *   c = (gamma - 1)/b2, dc/dbeta_k = beta_k (gamma^3 b2 - 2 (gamma - 1)) / b2^2, and
 *     dL_ij/dbeta_k = dc/dbeta_k beta_i beta_j + c (delta_ik beta_j + beta_i delta_jk),
 *     dL_it/dbeta_k = dL_ti/dbeta_k = gamma^3 beta_k beta_i + gamma delta_ik,
 *     dL_tt/dbeta_k = gamma^3 beta_k.
 * At beta = 0 the limits c = 1/2 and dc/dbeta = 0 are used. */
static void boost_grad_one(const double *vd, const double *betad, const double *gd, double *gv,
                           qreal *gbeta) {
  qreal L[4][4];
  if (!boost_matrix_q(betad, L)) {
    for (int k = 0; k < 4; k++) gv[k] = NAN;
    for (int k = 0; k < 3; k++) gbeta[k] = NAN;
    return;
  }
  qreal v[4], g[4], b[3];
  for (int k = 0; k < 4; k++) {
    v[k] = vd[k];
    g[k] = gd[k];
  }
  for (int k = 0; k < 3; k++) b[k] = betad[k];
  for (int j = 0; j < 4; j++) {
    qreal acc = 0;
    for (int i = 0; i < 4; i++) acc += L[i][j] * g[i];
    gv[j] = (double)acc;
  }
  qreal b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  qreal gam = 1 / Q_SQRT(1 - b2);
  qreal g3 = gam * gam * gam;
  qreal c = 0.5, dcf = 0; /* dc/dbeta_k = dcf * beta_k */
  if (b2 != 0) {
    c = (gam - 1) / b2;
    dcf = (g3 * b2 - 2 * (gam - 1)) / (b2 * b2);
  }
  for (int k = 0; k < 3; k++) {
    qreal dL[4][4];
    for (int i = 0; i < 3; i++) {
      for (int j = 0; j < 3; j++)
        dL[i][j] = dcf * b[k] * b[i] * b[j] + c * ((i == k ? b[j] : 0) + (j == k ? b[i] : 0));
      dL[i][3] = g3 * b[k] * b[i] + (i == k ? gam : 0);
      dL[3][i] = dL[i][3];
    }
    dL[3][3] = g3 * b[k];
    qreal acc = 0;
    for (int i = 0; i < 4; i++)
      for (int j = 0; j < 4; j++) acc += g[i] * dL[i][j] * v[j];
    gbeta[k] += acc;
  }
}

/* gv[i] = d<gout[i], out[i]>/dv[i];  gbeta[i] = d<gout[i], out[i]>/dbeta[i] for stride 1; for
 * stride 0 (one shared velocity) gbeta[0..2] is the sum over all i.  Single-threaded. */
void orc_boost_grad_def(const double *v, const double *beta, int64_t beta_stride,
                        const double *gout, int64_t n, double *gv, double *gbeta) {
  qreal shared[3] = {0, 0, 0};
  for (int64_t i = 0; i < n; i++) {
    if (beta_stride) {
      qreal gb[3] = {0, 0, 0};
      boost_grad_one(v + 4 * i, beta + 3 * i, gout + 4 * i, gv + 4 * i, gb);
      for (int k = 0; k < 3; k++) gbeta[3 * i + k] = (double)gb[k];
    } else {
      boost_grad_one(v + 4 * i, beta, gout + 4 * i, gv + 4 * i, shared);
    }
  }
  if (!beta_stride)
    for (int k = 0; k < 3; k++) gbeta[k] = (double)shared[k];
}

/* Jagged events (the per-event combinatorics of the RDataFrame analyses named as future work in
 * Sec. 6).  Event e owns particles [off[e], off[e+1]) (PtEtaPhiM rows).  Outputs:
 *   pair_off[e] = sum over earlier events of n(n-1)/2, pair_off[0] = 0 (n_events + 1 entries);
 *   pair_m[pair_off[e] + k(i,j)] = mass(p_i + p_j) for i < j, packed row-major:
 *     k(i,j) = i n - i(i+1)/2 + (j - i - 1);
 *   sums[e] = sum of the event's particles as PxPyPzE.
 * Returns 0, or -1 when the offsets are not a non-decreasing sequence starting at 0. */
int orc_event_pairs_def(const double *p, const int64_t *off, int64_t n_events, int64_t *pair_off,
                        double *pair_m, double *sums) {
  if (n_events < 0 || off[0] != 0) return -1;
  for (int64_t e = 0; e < n_events; e++)
    if (off[e + 1] < off[e]) return -1;
  pair_off[0] = 0;
  for (int64_t e = 0; e < n_events; e++) {
    int64_t n = off[e + 1] - off[e];
    pair_off[e + 1] = pair_off[e] + n * (n - 1) / 2;
  }
  for (int64_t e = 0; e < n_events; e++) {
    int64_t base = off[e], n = off[e + 1] - off[e];
    int64_t k = pair_off[e];
    for (int64_t i = 0; i < n; i++)
      for (int64_t j = i + 1; j < n; j++) pair_m[k++] = pair_mass_def(p + 4 * (base + i), p + 4 * (base + j));
    qreal s[4] = {0, 0, 0, 0};
    for (int64_t i = 0; i < n; i++) {
      qreal v[4];
      leg_to_cartesian_q(p + 4 * (base + i), v);
      for (int c = 0; c < 4; c++) s[c] += v[c];
    }
    for (int c = 0; c < 4; c++) sums[4 * e + c] = (double)s[c];
  }
  return 0;
}

/* Adjoint of orc_event_pairs_def (the per-event combinatorics, differentiated).  Inputs: the
 * upstream gradients gpm of the pair masses, packed as orc_event_pairs_def packs pair_m, and gsum
 * of the event sums (n_events rows of PxPyPzE; NULL means zero).  For particle i of event e:
 *   grad_p[i] = sum over j != i in e of gpm[pair(i, j)] dm(p_i, p_j)/dp_i  +  J_i^T gsum[e],
 * with pair(i, j) the packed index of the unordered pair and J_i the leg Jacobian above,
 * accumulated in binary128 and rounded once.  Returns 0, or -1 for malformed offsets. */
int orc_event_pairs_grad_def(const double *p, const int64_t *off, int64_t n_events,
                             const double *gpm, const double *gsum, double *grad_p) {
  if (n_events < 0 || off[0] != 0) return -1;
  for (int64_t e = 0; e < n_events; e++)
    if (off[e + 1] < off[e]) return -1;
  int64_t pbase = 0;  /* packed index of the event's first pair */
  for (int64_t e = 0; e < n_events; e++) {
    int64_t base = off[e], n = off[e + 1] - off[e];
    for (int64_t i = 0; i < n; i++) {
      const double *pi = p + 4 * (base + i);
      qreal acc[4] = {0, 0, 0, 0};
      for (int64_t j = 0; j < n; j++) {
        if (j == i) continue;
        int64_t lo = i < j ? i : j, hi = i < j ? j : i;
        int64_t k = lo * n - lo * (lo + 1) / 2 + (hi - lo - 1);
        qreal d[4], other[4];
        if (i < j)
          pair_mass_dm_q(pi, p + 4 * (base + j), d, other);
        else
          pair_mass_dm_q(p + 4 * (base + j), pi, other, d);
        for (int c = 0; c < 4; c++) acc[c] += (qreal)gpm[pbase + k] * d[c];
      }
      if (gsum) {
        qreal v[4], J[4][4];
        leg_to_cartesian_q(pi, v);
        leg_jacobian_q(pi, v, J);
        for (int c = 0; c < 4; c++)
          for (int r = 0; r < 4; r++) acc[c] += (qreal)gsum[4 * e + r] * J[r][c];
      }
      for (int c = 0; c < 4; c++) grad_p[4 * (base + i) + c] = (double)acc[c];
    }
    pbase += n * (n - 1) / 2;
  }
  return 0;
}

/* Fused per-event selection, pair-mass histogram and best candidate: the analysis step that the
 * per-event combinatorics serve (Sec. 6 names RDataFrame analyses as the next target; the paper
 * defines no such step, so its semantics are the ones written here).
 *   A particle passes when pt >= pt_min and |eta| <= eta_max.
 *   Every pair i < j of passing particles of an event has its mass m (the pair mass of Sec. 4.1,
 *   as in orc_event_pairs_def) counted in a histogram of n_bins equal bins over [lo, hi):
 *   counts[0] holds m < lo, counts[1 + b] the b-th bin, counts[n_bins + 1] m >= hi or NaN.
 *   The bin of m is floor((m - lo) * inv_w) with inv_w = n_bins / (hi - lo), both evaluated in
 *   double, and clamped to [0, n_bins - 1] (the clamp only acts on rounding at the upper edge).
 *   best_k[e] is the packed index k(i, j) (the order of orc_event_pairs_def) of the passing pair
 *   whose |m - target| is smallest, the smaller k on ties, or -1 when the event has no passing
 *   pair; best_m[e] is that pair's mass (NaN when none).
 * near_edge[s] counts the masses of slot s within rel_tol * max(|m|, |edge|) of one of the
 * slot's edges (lo + b (hi - lo) / n_bins, in double): another rounding of such an m may land
 * in the neighbouring slot.  Returns 0, or -1 for malformed offsets or n_bins < 1. */
int orc_pair_select_def(const double *p, const int64_t *off, int64_t n_events, double pt_min,
                        double eta_max, double lo, double hi, int32_t n_bins, double target,
                        double rel_tol, uint64_t *counts, uint64_t *near_edge, int64_t *best_k,
                        double *best_m) {
  if (n_events < 0 || off[0] != 0 || n_bins < 1 || !(hi > lo)) return -1;
  for (int64_t e = 0; e < n_events; e++)
    if (off[e + 1] < off[e]) return -1;
  for (int32_t s = 0; s < n_bins + 2; s++) counts[s] = near_edge[s] = 0;
  const double inv_w = (double)n_bins / (hi - lo);
  for (int64_t e = 0; e < n_events; e++) {
    const int64_t base = off[e], n = off[e + 1] - off[e];
    int64_t bk = -1;
    double bd = 0.0, bm = NAN;
    int64_t k = 0;
    for (int64_t i = 0; i < n; i++) {
      for (int64_t j = i + 1; j < n; j++, k++) {
        const double *a = p + 4 * (base + i), *b = p + 4 * (base + j);
        if (!(a[0] >= pt_min && fabs(a[1]) <= eta_max && b[0] >= pt_min && fabs(b[1]) <= eta_max))
          continue;
        const double m = pair_mass_def(a, b);
        int32_t slot;
        double e_lo, e_hi;  /* the slot's edges */
        if (m < lo) {
          slot = 0;
          e_lo = e_hi = lo;
        } else if (!(m < hi)) {
          slot = n_bins + 1;
          e_lo = e_hi = hi;
        } else {
          int64_t bin = (int64_t)floor((m - lo) * inv_w);
          if (bin < 0) bin = 0;
          if (bin > n_bins - 1) bin = n_bins - 1;
          slot = (int32_t)(bin + 1);
          e_lo = lo + (double)bin * (hi - lo) / n_bins;
          e_hi = lo + (double)(bin + 1) * (hi - lo) / n_bins;
        }
        counts[slot]++;
        if (m == m && (fabs(m - e_lo) <= rel_tol * fmax(fabs(m), fabs(e_lo)) ||
                       fabs(m - e_hi) <= rel_tol * fmax(fabs(m), fabs(e_hi))))
          near_edge[slot]++;
        const double d = fabs(m - target);
        if (d == d && (bk < 0 || d < bd)) {  /* strict: an equal later pair keeps the first */
          bk = k;
          bd = d;
          bm = m;
        }
      }
    }
    best_k[e] = bk;
    best_m[e] = bm;
  }
  return 0;
}

/* A general 4-D Lorentz transformation applied to PxPyPzE vectors (Sec. 4.1: transformations
 * are 4x4 matrices applied to every vector of an array; Sec. 3.1: vectors in any coordinate
 * system).  out[i] = L[i * l_stride] v[i], L row-major 4x4 in (x, y, z, t) order, evaluated in
 * binary128 and rounded once.  l_stride 0 applies one matrix to every vector.  The matrix is
 * taken as given (no check that it preserves the metric). */
void orc_lorentz_apply_def(const double *L16, int64_t l_stride, const double *v, int64_t n,
                           double *out) {
  for (int64_t i = 0; i < n; i++) {
    const double *L = L16 + 16 * l_stride * i;
    for (int r = 0; r < 4; r++) {
      qreal acc = 0;
      for (int k = 0; k < 4; k++) acc += (qreal)L[4 * r + k] * (qreal)v[4 * i + k];
      out[4 * i + r] = (double)acc;
    }
  }
}

/* A leg as PxPyPzE in binary128 (Sec. 3.1: any 4-D coordinate system): coords 0 gives
 * (px, py, pz, E) as stored; 1 gives (px, py, pz, m) with E = sqrt(px^2 + py^2 + pz^2 + m^2) (the
 * stored m enters through m^2); 2 gives (pt, eta, phi, E) with px = pt cos(phi), py = pt sin(phi),
 * pz = pt sinh(eta) and E as stored; 3 gives (pt, eta, phi, m) through leg_to_cartesian_q. */
static void cart_leg_q(const double *x, int coords, qreal out[4]) {
  if (coords == 3) {
    leg_to_cartesian_q(x, out);
    return;
  }
  if (coords == 2) {
    qreal pt = x[0], eta = x[1], phi = x[2];
    out[0] = pt * Q_COS(phi);
    out[1] = pt * Q_SIN(phi);
    out[2] = pt * Q_SINH(eta);
    out[3] = x[3];
    return;
  }
  out[0] = x[0];
  out[1] = x[1];
  out[2] = x[2];
  if (coords == 0) {
    out[3] = x[3];
  } else {
    qreal m = x[3];
    out[3] = Q_SQRT(out[0] * out[0] + out[1] * out[1] + out[2] * out[2] + m * m);
  }
}

/* Invariant mass of pairs given in any of the coordinate systems of cart_leg_q (Sec. 3.1: the
 * kernels are templated on the 4-D system; Sec. 4.1 Fig. 1 adds the pair and takes mass()):
 * m[i] = mass(a[i] + b[i]) with mass() as in lv_mass_q (a negative E^2 - |p|^2 gives -sqrt of its
 * magnitude, GenVector's convention for spacelike vectors). */
void orc_mass_cart_def(const double *a, const double *b, int64_t n, int coords, double *m) {
  for (int64_t i = 0; i < n; i++) {
    qreal va[4], vb[4], w[4];
    cart_leg_q(a + 4 * i, coords, va);
    cart_leg_q(b + 4 * i, coords, vb);
    for (int k = 0; k < 4; k++) w[k] = va[k] + vb[k];
    m[i] = (double)lv_mass_q(w);
  }
}

/* PtEtaPhiM -> PxPyPzE rounded to double (used by the tests to build boost inputs and
 * multi-body checks). */
void orc_to_cartesian_def(const double *p, int64_t n, double *out) {
  for (int64_t i = 0; i < n; i++) {
    qreal v[4];
    leg_to_cartesian_q(p + 4 * i, v);
    for (int c = 0; c < 4; c++) out[4 * i + c] = (double)v[c];
  }
}

/* Any coordinate system of cart_leg_q -> PxPyPzE, in binary128, rounded to double once. */
void orc_to_pxpypze_def(const double *p, int64_t n, int coords, double *out) {
  for (int64_t i = 0; i < n; i++) {
    qreal v[4];
    cart_leg_q(p + 4 * i, coords, v);
    for (int c = 0; c < 4; c++) out[4 * i + c] = (double)v[c];
  }
}

/* Mass of each PxPyPzE row, sqrt(E^2 - |p|^2) in binary128, rounded. */
void orc_lv_mass_def(const double *v, int64_t n, double *m) {
  for (int64_t i = 0; i < n; i++) {
    qreal w[4] = {v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]};
    m[i] = (double)lv_mass_q(w);
  }
}

/* ------------------------------------------------------------------------------------------ */
/* O2: cancellation-free identities in double                                                 */

/* Pair mass from non-negative terms only.  With P_i = pt_i cosh(eta_i) = |p_i| and
 * E_i = sqrt(P_i^2 + m_i^2):
 *   m^2 = m_1^2 + m_2^2 + 2 (E_1 E_2 - p_1.p_2)
 *   E_1 E_2 - P_1 P_2 = (m_1^2 P_2^2 + m_2^2 P_1^2 + m_1^2 m_2^2) / (E_1 E_2 + P_1 P_2)
 *   P_1 P_2 - p_1.p_2 = pt_1 pt_2 (cosh(d_eta) - cos(d_phi))
 *                     = 2 pt_1 pt_2 (sinh^2(d_eta/2) + sin^2(d_phi/2)).
 * Every term is >= 0 for pt >= 0, so the relative error is a few ulps. */
/* sin(d_phi / 2) up to sign, with d_phi = phi1 - phi2.  sin^2(d_phi/2) has period 2 pi, so for
 * |d_phi| > pi (both azimuths within [-pi, pi]) the half-angle is taken as
 * pi - |d_phi|/2 = ((pi - |phi1|) + (pi - |phi2|)) / 2: each bracket is an exact difference in
 * double (|phi| >= pi/2 there) and their sum has no cancellation, whereas phi1 - phi2 itself is
 * rounded to ~4e-16 absolute, which is a large relative error when |d_phi| is within ~1e-6 of
 * 2 pi. */
static double half_dphi_sin_fp64(double phi1, double phi2) {
  const double pid = 3.141592653589793116, pilo = 1.2246467991473531772e-16; /* pi = pid + pilo */
  double d = phi1 - phi2;
  if (fabs(d) > pid && fabs(phi1) <= pid && fabs(phi2) <= pid)
    return sin(0.5 * ((pid - fabs(phi1)) + (pid - fabs(phi2)) + 2.0 * pilo));
  return sin(0.5 * d);
}

static double pair_mass_fp64(const double *a, const double *b) {
  double pt1 = a[0], eta1 = a[1], phi1 = a[2], m1 = a[3];
  double pt2 = b[0], eta2 = b[1], phi2 = b[2], m2 = b[3];
  double P1 = pt1 * cosh(eta1), P2 = pt2 * cosh(eta2);
  double mm1 = m1 * m1, mm2 = m2 * m2;
  double E1 = sqrt(P1 * P1 + mm1), E2 = sqrt(P2 * P2 + mm2);
  double se = sinh(0.5 * (eta1 - eta2)), sp = half_dphi_sin_fp64(phi1, phi2);
  double t_mass = 2.0 * (mm1 * P2 * P2 + mm2 * P1 * P1 + mm1 * mm2) / (E1 * E2 + P1 * P2);
  double t_ang = 4.0 * pt1 * pt2 * (se * se + sp * sp);
  double denom = E1 * E2 + P1 * P2;
  if (denom == 0) t_mass = 0; /* both legs are zero vectors */
  return sqrt(mm1 + mm2 + t_mass + t_ang);
}

static void mass_fp64_range(void *p, int64_t lo, int64_t hi) {
  mass_ctx *c = (mass_ctx *)p;
  for (int64_t i = lo; i < hi; i++) c->m[i] = pair_mass_fp64(c->a + 4 * i, c->b + 4 * i);
}

void orc_mass_fp64(const double *a, const double *b, int64_t n, double *m, int nthreads) {
  mass_ctx c = {a, b, m};
  run_ranges(mass_fp64_range, &c, n, nthreads);
}

/* Adjoint of the O2 pair mass, from the same identity differentiated term by term.  With
 * F = m^2 = m_1^2 + m_2^2 + 2 Q + 4 pt_1 pt_2 S,  Q = E_1 E_2 - P_1 P_2,
 * S = sinh^2(d_eta/2) + sin^2(d_phi/2), dE_i/dP_i = P_i/E_i and dE_i/dm_i = m_i/E_i:
 *   dF/dP_1 = 2 (E_2 P_1 - P_2 E_1)/E_1 = 2 (P_1^2 m_2^2 - P_2^2 m_1^2) / (E_1 (E_2 P_1 + P_2 E_1))
 *     (the difference E_2 P_1 - P_2 E_1 multiplied by its conjugate), and likewise for leg 2;
 *   dF/dm_i = 2 m_i (E_1 + E_2)/E_i;
 *   dF/dpt_i = cosh(eta_i) dF/dP_i + 4 pt_o S;
 *   dF/deta_i = pt_i sinh(eta_i) dF/dP_i +- 2 pt_1 pt_2 sinh(d_eta);
 *   dF/dphi_i = +- 2 pt_1 pt_2 sin(d_phi)   (+ for leg 1, - for leg 2),
 * and dm/dx = dF/dx / (2 m).  sin(d_phi) = 2 sin(d_phi/2) cos(d_phi/2) from the half-angle of
 * half_dphi_sin_fp64 (for |d_phi| > pi its cosine changes sign).  Readings as O1's: where m = 0
 * the gradient is zero; a massless leg has E_i = P_i, so dE_i/dP_i = 1 and dF/dP_i =
 * 2 (E_o - P_o) = 2 m_o^2/(E_o + P_o), dF/dm_i = 0. */
static void half_dphi_sincos_fp64(double phi1, double phi2, double *sn, double *cs) {
  const double pid = 3.141592653589793116, pilo = 1.2246467991473531772e-16;
  double d = phi1 - phi2;
  if (fabs(d) > pid && fabs(phi1) <= pid && fabs(phi2) <= pid) {
    double h = 0.5 * ((pid - fabs(phi1)) + (pid - fabs(phi2)) + 2.0 * pilo); /* pi - |d|/2 */
    *sn = d > 0 ? sin(h) : -sin(h); /* sin(d/2) */
    *cs = -cos(h);                 /* cos(d/2) */
    return;
  }
  *sn = sin(0.5 * d);
  *cs = cos(0.5 * d);
}

static void pair_mass_dm_fp64(const double *a, const double *b, double ga[4], double gb[4]) {
  double pt[2] = {a[0], b[0]}, eta[2] = {a[1], b[1]}, mm[2] = {a[3], b[3]};
  double P[2], E[2], msq[2];
  for (int l = 0; l < 2; l++) {
    P[l] = pt[l] * cosh(eta[l]);
    msq[l] = mm[l] * mm[l];
    E[l] = sqrt(P[l] * P[l] + msq[l]);
  }
  double m = pair_mass_fp64(a, b);
  double *outs[2] = {ga, gb};
  if (!(m > 0)) {
    for (int l = 0; l < 2; l++)
      for (int k = 0; k < 4; k++) outs[l][k] = 0;
    return;
  }
  double de = eta[0] - eta[1];
  double se = sinh(0.5 * de), sp, cp;
  half_dphi_sincos_fp64(a[2], b[2], &sp, &cp);
  double S = se * se + sp * sp;
  double p12 = pt[0] * pt[1];
  double sinh_de = sinh(de), sin_dp = 2.0 * sp * cp;
  for (int l = 0; l < 2; l++) {
    int o = 1 - l;
    double dFdP, dFdm;
    if (mm[l] == 0) {
      dFdP = E[o] + P[o] > 0 ? 2.0 * msq[o] / (E[o] + P[o]) : 0.0;
      dFdm = 0.0;
    } else {
      double den = E[l] * (E[o] * P[l] + P[o] * E[l]);
      dFdP = den > 0 ? 2.0 * (P[l] * P[l] * msq[o] - P[o] * P[o] * msq[l]) / den : 0.0;
      dFdm = 2.0 * mm[l] * (E[0] + E[1]) / E[l];
    }
    double sgn = l == 0 ? 1.0 : -1.0;
    double dpt = cosh(eta[l]) * dFdP + 4.0 * pt[o] * S;
    double deta = pt[l] * sinh(eta[l]) * dFdP + sgn * 2.0 * p12 * sinh_de;
    double dphi = sgn * 2.0 * p12 * sin_dp;
    outs[l][0] = dpt / (2.0 * m);
    outs[l][1] = deta / (2.0 * m);
    outs[l][2] = dphi / (2.0 * m);
    outs[l][3] = dFdm / (2.0 * m);
  }
}

typedef struct {
  const double *a, *b, *gm;
  double *ga, *gb;
} mass_grad_fp64_ctx;

static void mass_grad_fp64_range(void *p, int64_t lo, int64_t hi) {
  mass_grad_fp64_ctx *c = (mass_grad_fp64_ctx *)p;
  for (int64_t i = lo; i < hi; i++) {
    double da[4], db[4];
    pair_mass_dm_fp64(c->a + 4 * i, c->b + 4 * i, da, db);
    for (int k = 0; k < 4; k++) {
      c->ga[4 * i + k] = c->gm[i] * da[k];
      c->gb[4 * i + k] = c->gm[i] * db[k];
    }
  }
}

/* O2 counterpart of orc_mass_grad_def. */
void orc_mass_grad_fp64(const double *a, const double *b, const double *gm, int64_t n,
                        double *ga, double *gb, int nthreads) {
  mass_grad_fp64_ctx c = {a, b, gm, ga, gb};
  run_ranges(mass_grad_fp64_range, &c, n, nthreads);
}

/* One leg as PxPyPzE in double: (pt cos phi, pt sin phi, pt sinh eta, sqrt((pt cosh eta)^2 + m^2)). */
static void leg_to_cartesian_fp64(const double *leg, double v[4]) {
  double pt = leg[0], eta = leg[1], phi = leg[2], mm = leg[3];
  double P = pt * cosh(eta);
  v[0] = pt * cos(phi);
  v[1] = pt * sin(phi);
  v[2] = pt * sinh(eta);
  v[3] = sqrt(P * P + mm * mm);
}

/* J^T g for one leg: g . dv/d(pt, eta, phi, m), v = leg_to_cartesian_fp64(leg); with
 * |J|^T |g| instead when magnitudes is set.  The derivatives of E are written with
 * E = sqrt(P^2 + m^2): dE/dpt = P cosh(eta)/E, dE/deta = P pt sinh(eta)/E, dE/dm = m/E, and for a
 * massless leg (E = P) cosh(eta) and pt sinh(eta), as in O1's reading. */
static void leg_jacobian_t_fp64(const double *leg, const double g[4], int magnitudes, double out[4]) {
  double pt = leg[0], eta = leg[1], phi = leg[2], mm = leg[3];
  double c = cos(phi), s = sin(phi), sh = sinh(eta), ch = cosh(eta);
  double P = pt * ch, E = sqrt(P * P + mm * mm);
  double J[4][4] = {{c, 0, -pt * s, 0}, {s, 0, pt * c, 0}, {sh, pt * ch, 0, 0}, {0, 0, 0, 0}};
  if (mm == 0) {
    J[3][0] = ch;
    J[3][1] = pt * sh;
  } else {
    J[3][0] = P * ch / E;
    J[3][1] = P * pt * sh / E;
    J[3][3] = mm / E;
  }
  for (int k = 0; k < 4; k++) {
    double acc = 0;
    for (int r = 0; r < 4; r++) acc += magnitudes ? fabs(g[r] * J[r][k]) : g[r] * J[r][k];
    out[k] = acc;
  }
}

typedef struct {
  const double *p;
  const int64_t *off, *pair_off;
  double *pair_m, *sums;
  const double *gpm, *gsum;
  double *grad_p;
  int magnitudes;
} event_fp64_ctx;

static void event_pairs_fp64_range(void *q, int64_t lo, int64_t hi) {
  event_fp64_ctx *c = (event_fp64_ctx *)q;
  for (int64_t e = lo; e < hi; e++) {
    int64_t base = c->off[e], n = c->off[e + 1] - c->off[e], k = c->pair_off[e];
    for (int64_t i = 0; i < n; i++)
      for (int64_t j = i + 1; j < n; j++)
        c->pair_m[k++] = pair_mass_fp64(c->p + 4 * (base + i), c->p + 4 * (base + j));
    double s[4] = {0, 0, 0, 0};
    for (int64_t i = 0; i < n; i++) {
      double v[4];
      leg_to_cartesian_fp64(c->p + 4 * (base + i), v);
      for (int r = 0; r < 4; r++) s[r] += v[r];
    }
    for (int r = 0; r < 4; r++) c->sums[4 * e + r] = s[r];
  }
}

static int check_offsets(const int64_t *off, int64_t n_events) {
  if (n_events < 0 || off[0] != 0) return -1;
  for (int64_t e = 0; e < n_events; e++)
    if (off[e + 1] < off[e]) return -1;
  return 0;
}

/* O2 counterpart of orc_event_pairs_def (same packing and outputs): pair masses by the O2
 * identity, event sums accumulated in double; events split over nthreads threads. */
int orc_event_pairs_fp64(const double *p, const int64_t *off, int64_t n_events, int64_t *pair_off,
                         double *pair_m, double *sums, int nthreads) {
  if (check_offsets(off, n_events)) return -1;
  pair_off[0] = 0;
  for (int64_t e = 0; e < n_events; e++) {
    int64_t n = off[e + 1] - off[e];
    pair_off[e + 1] = pair_off[e] + n * (n - 1) / 2;
  }
  event_fp64_ctx c = {p, off, pair_off, pair_m, sums, NULL, NULL, NULL, 0};
  run_ranges(event_pairs_fp64_range, &c, n_events, nthreads);
  return 0;
}

static void event_pairs_grad_fp64_range(void *q, int64_t lo, int64_t hi) {
  event_fp64_ctx *c = (event_fp64_ctx *)q;
  for (int64_t e = lo; e < hi; e++) {
    int64_t base = c->off[e], n = c->off[e + 1] - c->off[e], pbase = c->pair_off[e];
    for (int64_t i = 0; i < n; i++) {
      const double *pi = c->p + 4 * (base + i);
      double acc[4] = {0, 0, 0, 0};
      for (int64_t j = 0; j < n; j++) {
        if (j == i) continue;
        int64_t a = i < j ? i : j, b = i < j ? j : i;
        int64_t k = a * n - a * (a + 1) / 2 + (b - a - 1);
        double d[4], other[4];
        if (i < j)
          pair_mass_dm_fp64(pi, c->p + 4 * (base + j), d, other);
        else
          pair_mass_dm_fp64(c->p + 4 * (base + j), pi, other, d);
        for (int r = 0; r < 4; r++)
          acc[r] += c->magnitudes ? fabs(c->gpm[pbase + k] * d[r]) : c->gpm[pbase + k] * d[r];
      }
      if (c->gsum) {
        double t[4];
        leg_jacobian_t_fp64(pi, c->gsum + 4 * e, c->magnitudes, t);
        for (int r = 0; r < 4; r++) acc[r] += t[r];
      }
      for (int r = 0; r < 4; r++) c->grad_p[4 * (base + i) + r] = acc[r];
    }
  }
}

/* O2 counterpart of orc_event_pairs_grad_def (same inputs and packing; gsum may be NULL), in
 * double; with magnitudes set, the per-particle sums of the contributions' magnitudes instead
 * (|gpm| |dm/dp| over the particle's pairs plus |J|^T |gsum|): the scale that a correct
 * summation in any order reaches, used to bound an adjoint's error. */
int orc_event_pairs_grad_fp64(const double *p, const int64_t *off, int64_t n_events,
                              const double *gpm, const double *gsum, int magnitudes,
                              double *grad_p, int nthreads) {
  if (check_offsets(off, n_events)) return -1;
  int64_t *pair_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_events + 1));
  if (!pair_off) return -2;
  pair_off[0] = 0;
  for (int64_t e = 0; e < n_events; e++) {
    int64_t n = off[e + 1] - off[e];
    pair_off[e + 1] = pair_off[e] + n * (n - 1) / 2;
  }
  event_fp64_ctx c = {p, off, pair_off, NULL, NULL, gpm, gsum, grad_p, magnitudes};
  run_ranges(event_pairs_grad_fp64_range, &c, n_events, nthreads);
  free(pair_off);
  return 0;
}

/* Boost in vector form:
 *   E' = gamma (E + beta.p),  p' = p + (k (beta.p) + gamma E) beta,  k = gamma^2 / (1 + gamma),
 * using (gamma - 1)/b2 = gamma^2/(1 + gamma), which has no 0/0 at beta = 0. */
static void boost_fp64_range(void *p, int64_t lo, int64_t hi) {
  boost_ctx *c = (boost_ctx *)p;
  for (int64_t i = lo; i < hi; i++) {
    const double *vi = c->v + 4 * i, *bi = c->beta + 3 * c->stride * i;
    double *oi = c->out + 4 * i;
    double b2 = bi[0] * bi[0] + bi[1] * bi[1] + bi[2] * bi[2];
    if (!(b2 < 1)) {
      for (int k = 0; k < 4; k++) oi[k] = NAN;
      continue;
    }
    double g = 1.0 / sqrt(1.0 - b2);
    double k = g * g / (1.0 + g);
    double bp = bi[0] * vi[0] + bi[1] * vi[1] + bi[2] * vi[2];
    double f = k * bp + g * vi[3];
    oi[0] = vi[0] + f * bi[0];
    oi[1] = vi[1] + f * bi[1];
    oi[2] = vi[2] + f * bi[2];
    oi[3] = g * (vi[3] + bp);
  }
}

void orc_boost_fp64(const double *v, const double *beta, int64_t beta_stride, int64_t n,
                    double *out, int nthreads) {
  boost_ctx c = {v, beta, beta_stride, out};
  run_ranges(boost_fp64_range, &c, n, nthreads);
}
