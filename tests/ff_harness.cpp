// Host build of the library's float-float arithmetic (paper_2312_02756_gb300/csrc/ff.cuh and
// mass_ff.cuh) for the CPU tests: the same source the kernels compile, called over arrays.
#include <math.h>
#include <stdint.h>

#include "../paper_2312_02756_gb300/csrc/ff.cuh"
#include "../paper_2312_02756_gb300/csrc/mass_ff.cuh"
#include "../paper_2312_02756_gb300/csrc/boost_ff.cuh"
#include "../paper_2312_02756_gb300/csrc/cart_mass.cuh"
#include "../paper_2312_02756_gb300/csrc/cart_fixed.cuh"
#include "../paper_2312_02756_gb300/csrc/apply_ff.cuh"
#include "../paper_2312_02756_gb300/csrc/convert_ff.cuh"
#include "../paper_2312_02756_gb300/csrc/mass_ff2.cuh"
#include "../paper_2312_02756_gb300/csrc/mass_lc.cuh"
#include "../paper_2312_02756_gb300/csrc/mass_lc_grad.cuh"
#include "../paper_2312_02756_gb300/csrc/ptetaphie_lc.cuh"

using namespace gvx::ffm;

static TabRef tables() { return TabRef{kExpTab, kTrigTab}; }

extern "C" {

int64_t ffh_mass(const double *a, const double *b, int64_t n, double *m, uint8_t *ok) {
  int64_t c = 0;
  for (int64_t i = 0; i < n; i++) {
    const double *x = a + 4 * i, *y = b + 4 * i;
    double out = NAN;
    bool f = pair_mass_ff(x[0], x[1], x[2], x[3], y[0], y[1], y[2], y[3], tables(), &out);
    ok[i] = f;
    m[i] = out;
    c += f;
  }
  return c;
}

// The light-cone fast path of the FP64 mass kernel (mass_lc.cuh).
int64_t ffh_mass_lc(const double *a, const double *b, int64_t n, double *m, uint8_t *ok) {
  int64_t c = 0;
  const LcTab T{kHypTab, kSinTab};
  for (int64_t i = 0; i < n; i++) {
    const double *x = a + 4 * i, *y = b + 4 * i;
    double out = NAN;
    bool f = pair_mass_lc(x[0], x[1], x[2], x[3], y[0], y[1], y[2], y[3], T, &out);
    ok[i] = f;
    m[i] = out;
    c += f;
  }
  return c;
}

// The jagged kernel's route for the same pairs: each particle's light-cone terms computed alone
// (scalar) at the scale of the larger high word of (pt, |m|) over both legs and `extra` (an
// event's other particles), then the shared pair step and the integer-assembled output.
// ok[i] = 0 where either route declines.
int64_t ffh_mass_lc_event(const double *a, const double *b, const double *extra, int64_t n,
                          double *m, uint8_t *ok) {
  int64_t c = 0;
  const LcTab T{kHypTab, kSinTab};
  for (int64_t i = 0; i < n; i++) {
    const double *x = a + 4 * i, *y = b + 4 * i;
    uint32_t w = umax32(umax32(dhi(x[0]), dhi(x[3]) & 0x7fffffffu), umax32(dhi(y[0]), dhi(y[3]) & 0x7fffffffu));
    w = umax32(w, umax32(dhi(extra[i]), 0u));
    const uint32_t ew = w & 0x7ff00000u, rb = ew - (127u << 20);
    ff pt[2], Y[2], D[2];
    for (int l = 0; l < 2; l++) {
      const double *v = l ? y : x;
      const ff ptf = cvt1(cvt_parts(dhi(v[0]), dlo(v[0]), rb));
      const ff mmf = cvt1(cvt_parts(dhi(v[3]) & 0x7fffffffu, dlo(v[3]), rb));
      const ff xe = cvt1(cvt_parts(umax32(dhi(v[1]) & 0x7fffffffu, 0x3E100000u), dlo(v[1]), kRebaseOne));
      const LcLeg<ff> L = lc_leg(ptf, mmf, xe, T.hyp);
      pt[l] = ptf;
      Y[l] = L.Y;
      D[l] = L.D;
    }
    ff S, m2s;
    const bool oks = lc_pair_S(x[1], y[1], x[2], y[2], T, &S);
    bool f = lc_pair_m2(pt[0], pt[1], Y[0], Y[1], D[0], D[1], S, &m2s) && oks;
    ok[i] = f;
    m[i] = f ? lc_mass_out_int(m2s, ew) : NAN;
    c += f;
  }
  return c;
}

int64_t ffh_mass_grad(const double *a, const double *b, const double *gm, int64_t n, double *ga,
                      double *gb, uint8_t *ok) {
  int64_t c = 0;
  for (int64_t i = 0; i < n; i++) {
    const double *x = a + 4 * i, *y = b + 4 * i;
    double out[8];
    bool f = pair_mass_grad_ff(x[0], x[1], x[2], x[3], y[0], y[1], y[2], y[3], gm[i], tables(),
                               out);
    ok[i] = f;
    for (int k = 0; k < 4; k++) {
      ga[4 * i + k] = f ? out[k] : NAN;
      gb[4 * i + k] = f ? out[4 + k] : NAN;
    }
    c += f;
  }
  return c;
}

// The light-cone adjoint of the FP64 mass kernel (mass_lc_grad.cuh); ms = nullptr: no saved
// masses (the forward's m is recomputed).
int64_t ffh_mass_grad_lc(const double *a, const double *b, const double *gm, const double *ms,
                         int64_t n, double *ga, double *gb, uint8_t *ok) {
  int64_t c = 0;
  const LcTab T{kHypTab, kSinTab};
  for (int64_t i = 0; i < n; i++) {
    const double *x = a + 4 * i, *y = b + 4 * i;
    double out[8];
    bool f = pair_mass_grad_lc(x[0], x[1], x[2], x[3], y[0], y[1], y[2], y[3], gm[i],
                               ms != nullptr, ms ? ms[i] : 0.0, T, out);
    ok[i] = f;
    for (int k = 0; k < 4; k++) {
      ga[4 * i + k] = f ? out[k] : NAN;
      gb[4 * i + k] = f ? out[4 + k] : NAN;
    }
    c += f;
  }
  return c;
}

// The light-cone PtEtaPhiE pair mass of the FP64 kernel (ptetaphie_lc.cuh).
int64_t ffh_mass_e_lc(const double *a, const double *b, int64_t n, double *m, uint8_t *ok) {
  int64_t c = 0;
  const LcTab T{kHypTab, kSinTab};
  for (int64_t i = 0; i < n; i++) {
    const double *x = a + 4 * i, *y = b + 4 * i;
    double out = NAN;
    ok[i] = pair_mass_e_lc(x[0], x[1], x[2], x[3], y[0], y[1], y[2], y[3], T, &out);
    m[i] = out;
    c += ok[i];
  }
  return c;
}

// lc_to_double_int of the ff (hi[i], lo[i]) times 2^shift (mass_lc.cuh)
void ffh_lc_to_double_int(const float *hi, const float *lo, int64_t n, int shift, double *out) {
  for (int64_t i = 0; i < n; i++)
    out[i] = lc_to_double_int(ff{hi[i], lo[i]}, (uint32_t)(896 + shift) << 20);
}

// lc_to_double of the ff (hi[i], lo[i]) times 2^shift (mass_lc.cuh)
void ffh_lc_to_double(const float *hi, const float *lo, int64_t n, int shift, double *out) {
  for (int64_t i = 0; i < n; i++) out[i] = lc_to_double(ff{hi[i], lo[i]}, (uint32_t)(896 + shift) << 20);
}

// op: 0 cosh, 1 sinh, 2 sin_q1, 3 round trip double -> ff -> double, 4 sqrt, 5 sqr
void ffh_unary(int op, const double *x, int64_t n, double *out, uint8_t *ok) {
  for (int64_t i = 0; i < n; i++) {
    bool f = true;
    ff v = from_double(x[i], &f);
    ff r;
    switch (op) {
      case 0: r = cosh_t(v, tables()); break;
      case 1: r = sinh_t(v, tables()); break;
      case 2: r = sin_t(v, tables()); break;
      case 3: r = v; break;
      case 4: r = sqrt(v); break;
      default: r = sqr(v); break;
    }
    out[i] = to_double(r);
    ok[i] = f;
  }
}

// gamma = 1/sqrt(1 - b2) and w = gamma/(1 + gamma) as the FP64 boost computes them.
void ffh_boost_coef(const double *beta, int64_t n, double *g, double *w, uint8_t *ok) {
  for (int64_t i = 0; i < n; i++) {
    bool f = true;
    ff omb = one_minus_sq3(beta[3 * i], beta[3 * i + 1], beta[3 * i + 2], &f);
    ff s = sqrt(omb);
    ff gg = recip(s);
    ff ww = recip(add_same(make(1.0f), s));
    g[i] = to_double(gg);
    w[i] = to_double(ww);
    ok[i] = f;
  }
}

// from_double_ranged(x, shift) as (hi, lo) doubles, with same[i] = 1 where it is bitwise
// from_double(x, shift), 0 where it differs, 2 where from_double rejects x.
void ffh_conv_ranged(const double *x, int64_t n, int shift, double *hi, double *lo,
                     uint8_t *same) {
  for (int64_t i = 0; i < n; i++) {
    bool f = true;
    ff a = from_double(x[i], &f, shift);
    ff b = from_double_ranged(x[i], shift);
    hi[i] = b.hi;
    lo[i] = b.lo;
    uint32_t ah = f2u(a.hi), al = f2u(a.lo), bh = f2u(b.hi), bl = f2u(b.lo);
    same[i] = !f ? 2 : (ah == bh && al == bl) ? 1 : 0;
  }
}

// The FP64 boost adjoint's fast path: v (n, 4), beta (n, 3), grad_out (n, 4) -> gv (n, 4),
// gbeta (n, 3); ok[i] = in domain.
int64_t ffh_boost_bwd(const double *v, const double *beta, const double *gout, int64_t n,
                      double *gv, double *gbeta, uint8_t *ok) {
  int64_t c = 0;
  for (int64_t i = 0; i < n; i++) {
    const double *b = beta + 3 * i;
    const BetaBwdFF B = beta_bwd_ff(b[0], b[1], b[2]);
    bool f = boost_bwd_ff(B, b[0], b[1], b[2], v + 4 * i, gout + 4 * i, gv + 4 * i, gbeta + 3 * i);
    if (!f) {
      for (int k = 0; k < 4; k++) gv[4 * i + k] = NAN;
      for (int k = 0; k < 3; k++) gbeta[3 * i + k] = NAN;
    }
    ok[i] = f;
    c += f;
  }
  return c;
}

// The Cartesian pair mass (FP64): a, b (n, 4) with coords 0 (E stored) or 1 (m stored).
int64_t ffh_mass_cart(const double *a, const double *b, int64_t n, int coords, double *m,
                      uint8_t *ok) {
  int64_t c = 0;
  for (int64_t i = 0; i < n; i++) {
    m[i] = gvx::cart::mass(a + 4 * i, b + 4 * i, coords);
    ok[i] = 1;
    c += 1;
  }
  return c;
}

// The fixed-point fast paths of the Cartesian pair mass (coords 0: PxPyPzE, 1: PxPyPzM): FP64
// legs (m) and the same legs rounded to float (m32); ok / ok32 = inside the fast path.
int64_t ffh_mass_cart_fixed(const double *a, const double *b, int64_t n, int coords, double *m,
                            uint8_t *ok, float *m32, uint8_t *ok32) {
  int64_t c = 0;
  for (int64_t i = 0; i < n; i++) {
    double out = NAN;
    ok[i] = coords == 0 ? gvx::cfix::mass_pxpypze(a + 4 * i, b + 4 * i, &out)
                        : gvx::cfix::mass_pxpypzm(a + 4 * i, b + 4 * i, &out);
    m[i] = out;
    c += ok[i];
    float fa[4], fb[4], o32 = NAN;
    for (int k = 0; k < 4; k++) {
      fa[k] = (float)a[4 * i + k];
      fb[k] = (float)b[4 * i + k];
    }
    ok32[i] = coords == 0 ? gvx::cfix::mass_pxpypze(fa, fb, &o32) : gvx::cfix::mass_pxpypzm(fa, fb, &o32);
    m32[i] = o32;
  }
  return c;
}

// The float-float Lorentz transformation with one shared matrix L (16, row-major): v, out (n, 4);
// returns -1 when L is outside the domain, else the number of vectors taken (ok[i]).
int64_t ffh_apply(const double *L, const double *v, int64_t n, double *out, uint8_t *ok) {
  const LorentzFF M = lorentz_ff(L);
  if (!M.ok) return -1;
  ff2 lp[8];
  pair_rows(M, lp);
  int64_t c = 0;
  for (int64_t i = 0; i < n; i++) {
    ok[i] = apply_ff(lp, M.r, v + 4 * i, out + 4 * i);
    c += ok[i];
  }
  return c;
}

// The float-float conversion to PxPyPzE: coords 0 PtEtaPhiM, 2 PxPyPzM, 3 PtEtaPhiE (the library's
// gvx_coords codes); p, out (n, 4); ok[i] = inside the fast path.
int64_t ffh_convert(const double *p, int64_t n, int coords, double *out, uint8_t *ok) {
  int64_t c = 0;
  const LcTab T{kHypTab, kSinTab};
  for (int64_t i = 0; i < n; i++) {
    const double *x = p + 4 * i;
    double *o = out + 4 * i;
    ok[i] = coords == 2 ? pxpypzm_to_cart(x, o)
                        : ptetaphi_to_cart_lc(x[0], x[1], x[2], x[3], coords == 3, T, o);
    c += ok[i];
  }
  return c;
}

// The pair mass with its two legs paired (pair_mass_ff_lp).
int64_t ffh_mass_lp(const double *a, const double *b, int64_t n, double *m, uint8_t *ok) {
  int64_t c = 0;
  for (int64_t i = 0; i < n; i++) {
    const double *x = a + 4 * i, *y = b + 4 * i;
    double out = NAN;
    ok[i] = pair_mass_ff_lp(x[0], x[1], x[2], x[3], y[0], y[1], y[2], y[3], tables(), &out);
    m[i] = out;
    c += ok[i];
  }
  return c;
}

// to_double_int and the FP64-add conversion to_double of the ff values (hi[i], lo[i]) * 2^shift.
void ffh_to_double(const float *hi, const float *lo, int64_t n, int shift, double *out_int,
                   double *out_add) {
  for (int64_t i = 0; i < n; i++) {
    out_int[i] = to_double_int(ff{hi[i], lo[i]}, shift);
    out_add[i] = to_double(ff{hi[i], lo[i]}, shift);
  }
}

// The FP64 boost's fast path: v (n, 4) PxPyPzE, beta (n, 3) -> out (n, 4), ok[i] = in domain.
int64_t ffh_boost(const double *v, const double *beta, int64_t n, double *out, uint8_t *ok) {
  int64_t c = 0;
  for (int64_t i = 0; i < n; i++) {
    const double *x = v + 4 * i, *b = beta + 3 * i;
    const BetaFF B = beta_ff(b[0], b[1], b[2]);
    bool f = boost_ff(B, b[0], b[1], b[2], x[0], x[1], x[2], x[3], out + 4 * i);
    if (!f)
      for (int k = 0; k < 4; k++) out[4 * i + k] = NAN;
    ok[i] = f;
    c += f;
  }
  return c;
}

// op: 0 exact difference, 1 mul, 2 div, 3 add
void ffh_binary(int op, const double *x, const double *y, int64_t n, double *out, uint8_t *ok) {
  for (int64_t i = 0; i < n; i++) {
    bool f = true;
    ff r;
    if (op == 0) {
      r = from_double(x[i] - y[i], &f);
    } else {
      ff a = from_double(x[i], &f), b = from_double(y[i], &f);
      r = op == 1 ? mul(a, b) : op == 2 ? div(a, b) : add(a, b);
    }
    out[i] = to_double(r);
    ok[i] = f;
  }
}
}
