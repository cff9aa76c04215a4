/*
 * Plain C statement of the oracle's EFIE entry (oracle/efie.py), used by the
 * oracle's ACA to evaluate single rows and columns without interpreter
 * overhead.  TEST INFRASTRUCTURE: part of the CPU oracle, never linked into
 * the GPU library.
 *
 *   Z_mn = j eta sum_{a in T_m+-, b in T_n+-} s_a s_b l_m l_n [(k/4) A_ij - S0/k]
 *   A_ij = S3 - (S2 . v_j + v_i . S1) + (v_i . v_j) S0
 * S0..S3: normalised 7x7-point sums of G = e^{-jkR}/(4 pi R) (Eq. 3 with the
 * e^{+jwt} convention); on triangle pairs sharing a vertex G - 1/(4 pi R) is
 * summed and the 1/(4 pi R) part integrated in closed form over the
 * higher-index triangle (Wilton et al. 1984 / Graglia 1993), the inner and
 * outer first moments of a self pair averaged.
 */
#include <math.h>
#include <stddef.h>

typedef struct {
  const double* V;     /* nv x 3 */
  const long long* T;  /* nt x 3 */
  const double* Q;     /* nt x 7 x 3 quadrature points */
  const double* area;  /* nt */
  const long long* tp; /* N: T+ */
  const long long* tm; /* N: T- */
  const long long* fp; /* N: local free vertex in T+ */
  const long long* fm; /* N: local free vertex in T- */
  const double* len;   /* N */
  const double* w;     /* 7 weights */
  double k, eta;
} mesh_t;

static void sub3(const double* a, const double* b, double* o) {
  o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2];
}
static double dot3(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void cross3(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

/* int_T 1/R ds' and int_T (r' - rho)/R ds' (closed form). */
static void static_pot(const double* r, const double* p0, const double* p1, const double* p2,
                       double* Is, double* Iv, double* rho) {
  double e1[3], e2[3], n[3];
  sub3(p1, p0, e1);
  sub3(p2, p0, e2);
  cross3(e1, e2, n);
  double nn = sqrt(dot3(n, n));
  n[0] /= nn; n[1] /= nn; n[2] /= nn;
  double d[3];
  sub3(r, p0, d);
  double h = dot3(n, d);
  for (int c = 0; c < 3; ++c) rho[c] = r[c] - h * n[c];
  double ah = fabs(h);
  const double* P[3] = {p0, p1, p2};
  *Is = 0.0;
  Iv[0] = Iv[1] = Iv[2] = 0.0;
  for (int e = 0; e < 3; ++e) {
    const double* pa = P[e];
    const double* pb = P[(e + 1) % 3];
    double ed[3], lh[3], uh[3], t1[3], t2[3];
    sub3(pb, pa, ed);
    double elen = sqrt(dot3(ed, ed));
    for (int c = 0; c < 3; ++c) lh[c] = ed[c] / elen;
    cross3(lh, n, uh);
    sub3(pb, rho, t1);
    sub3(pa, rho, t2);
    double lp = dot3(t1, lh), lm = dot3(t2, lh), t = dot3(t2, uh);
    double R0sq = t * t + h * h;
    double Rp = sqrt(R0sq + lp * lp), Rm = sqrt(R0sq + lm * lm);
    double f = 0.0, beta = 0.0;
    if (!(R0sq <= (1e-14 * elen) * (1e-14 * elen))) {
      f = (lm + lp >= 0.0) ? log((Rp + lp) / (Rm + lm)) : log((Rm - lm) / (Rp - lp));
      if (ah > 0.0) beta = atan(t * lp / (R0sq + ah * Rp)) - atan(t * lm / (R0sq + ah * Rm));
    }
    *Is += t * f - ah * beta;
    double cc = 0.5 * (R0sq * f + lp * Rp - lm * Rm);
    for (int c = 0; c < 3; ++c) Iv[c] += uh[c] * cc;
  }
}

/* S[0] = S0, S[1..3] = S1, S[4..6] = S2, S[7] = S3, each (re, im). */
static void pair_moments(const mesh_t* M, long long a, long long b, double S[8][2]) {
  const long long* ta = M->T + 3 * a;
  const long long* tb = M->T + 3 * b;
  int touch = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) touch |= (ta[i] == tb[j]);
  for (int i = 0; i < 8; ++i) S[i][0] = S[i][1] = 0.0;
  const double inv4pi = 1.0 / (4.0 * M_PI);
  for (int p = 0; p < 7; ++p) {
    const double* rp = M->Q + (a * 7 + p) * 3;
    for (int q = 0; q < 7; ++q) {
      const double* rq = M->Q + (b * 7 + q) * 3;
      double d[3];
      sub3(rp, rq, d);
      double R = sqrt(dot3(d, d));
      double gr, gi;
      if (R == 0.0) {
        gr = 0.0;
        gi = -M->k * inv4pi;
      } else {
        double c = cos(M->k * R), s = sin(M->k * R);
        gr = (touch ? c - 1.0 : c) * inv4pi / R;
        gi = -s * inv4pi / R;
      }
      double ww = M->w[p] * M->w[q];
      gr *= ww;
      gi *= ww;
      double pq = dot3(rp, rq);
      S[0][0] += gr; S[0][1] += gi;
      for (int c = 0; c < 3; ++c) {
        S[1 + c][0] += gr * rq[c]; S[1 + c][1] += gi * rq[c];
        S[4 + c][0] += gr * rp[c]; S[4 + c][1] += gi * rp[c];
      }
      S[7][0] += gr * pq; S[7][1] += gi * pq;
    }
  }
  if (touch) {
    long long lo = a < b ? a : b, hi = a < b ? b : a;
    const long long* th = M->T + 3 * hi;
    const double *p0 = M->V + 3 * th[0], *p1 = M->V + 3 * th[1], *p2 = M->V + 3 * th[2];
    double s0 = 0, s3 = 0, sin_[3] = {0, 0, 0}, sout[3] = {0, 0, 0};
    for (int p = 0; p < 7; ++p) {
      const double* ro = M->Q + (lo * 7 + p) * 3;
      double Is, Iv[3], rh[3];
      static_pot(ro, p0, p1, p2, &Is, Iv, rh);
      double Jv[3] = {Iv[0] + rh[0] * Is, Iv[1] + rh[1] * Is, Iv[2] + rh[2] * Is};
      double sc = M->w[p] / (4.0 * M_PI * M->area[hi]);
      s0 += sc * Is;
      for (int c = 0; c < 3; ++c) {
        sin_[c] += sc * Jv[c];
        sout[c] += sc * Is * ro[c];
      }
      s3 += sc * dot3(ro, Jv);
    }
    if (a == b)
      for (int c = 0; c < 3; ++c) sin_[c] = sout[c] = 0.5 * (sin_[c] + sout[c]);
    const double* m1 = (a > b) ? sout : sin_;
    const double* m2 = (a > b) ? sin_ : sout;
    S[0][0] += s0;
    S[7][0] += s3;
    for (int c = 0; c < 3; ++c) {
      S[1 + c][0] += m1[c];
      S[4 + c][0] += m2[c];
    }
  }
}

static void entry(const mesh_t* M, long long m, long long n, double* out) {
  double t[2][2][2];
  const long long* tri[2] = {M->tp, M->tm};
  const long long* fv[2] = {M->fp, M->fm};
  for (int sa = 0; sa < 2; ++sa) {
    long long a = tri[sa][m];
    const double* va = M->V + 3 * M->T[3 * a + fv[sa][m]];
    for (int sb = 0; sb < 2; ++sb) {
      long long b = tri[sb][n];
      const double* vb = M->V + 3 * M->T[3 * b + fv[sb][n]];
      double S[8][2];
      pair_moments(M, a, b, S);
      double vv = dot3(va, vb);
      double sg = (sa == sb) ? 1.0 : -1.0;
      double ll = M->len[m] * M->len[n] * sg;
      for (int c = 0; c < 2; ++c) {
        double s2v = S[4][c] * vb[0] + S[5][c] * vb[1] + S[6][c] * vb[2];
        double vs1 = va[0] * S[1][c] + va[1] * S[2][c] + va[2] * S[3][c];
        double A = S[7][c] - (s2v + vs1) + vv * S[0][c];
        t[sa][sb][c] = ll * ((M->k / 4.0) * A - S[0][c] / M->k);
      }
    }
  }
  double zr = (t[0][0][0] + t[1][1][0]) + (t[0][1][0] + t[1][0][0]);
  double zi = (t[0][0][1] + t[1][1][1]) + (t[0][1][1] + t[1][0][1]);
  out[0] = -M->eta * zi;    /* j eta z */
  out[1] = M->eta * zr;
}

/* out (nrows x ncols complex, row-major, interleaved) = Z[rows][cols] */
void efie_block_c(const double* V, const long long* T, const double* Q, const double* area,
                  const long long* tp, const long long* tm, const long long* fp,
                  const long long* fm, const double* len, const double* w, double k, double eta,
                  long long nrows, const long long* rows, long long ncols, const long long* cols,
                  double* out) {
  mesh_t M = {V, T, Q, area, tp, tm, fp, fm, len, w, k, eta};
  for (long long i = 0; i < nrows; ++i)
    for (long long j = 0; j < ncols; ++j) entry(&M, rows[i], cols[j], out + 2 * (i * ncols + j));
}
