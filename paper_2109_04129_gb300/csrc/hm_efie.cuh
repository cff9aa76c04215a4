// Device-side EFIE Galerkin entry of two RWG functions (Eq. 2-3, time
// convention e^{+jwt}, G = e^{-jkR}/(4 pi R)):
//   Z_mn = j eta * sum_{a in T_m+-, b in T_n+-} s_a s_b l_m l_n [ (k/4) A_ij - S0 / k ]
//   A_ij = S3 - (S2 . v_j + v_i . S1) + (v_i . v_j) S0
// with the normalised 7x7-point pair sums S0 = sum w_p w_q G, S1 = sum w w G r_q,
// S2 = sum w w G r_p, S3 = sum w w G (r_p . r_q) and v_i, v_j the free
// vertices.  Pairs sharing a vertex take the static part 1/(4 pi R) in closed
// form over the higher-index triangle (outer points on the lower-index one)
// and the remainder (e^{-jkR} - 1)/(4 pi R) by quadrature; on a self pair the
// inner and outer first moments are averaged.
#pragma once
#include "hm_internal.h"

namespace hm {

struct MeshDev {
  const double* V;      // nv x 3 vertices
  const int* T;         // nt x 3 triangles
  const double* Q;      // nt x 7 x 3 quadrature points
  const double* area;   // nt
  const int* tri[2];    // RWG -> T+ / T-
  const int* fv[2];     // RWG -> local index of the free vertex in T+ / T-
  const double* len;    // RWG edge length
  double k, eta;
};

// Symmetric 7-point degree-5 rule: weights (centroid, orbit a1 x3, orbit a2 x3).
__device__ __forceinline__ double qw(int q) {
  // (155 -+ sqrt 15)/1200, 9/40
  const double s15 = 3.872983346207417;   // sqrt(15)
  return q == 0 ? 9.0 / 40.0 : (q <= 3 ? (155.0 - s15) / 1200.0 : (155.0 + s15) / 1200.0);
}

struct V3 { double x, y, z; };
__device__ __forceinline__ V3 v3(const double* p) { return V3{p[0], p[1], p[2]}; }
__device__ __forceinline__ V3 sub(V3 a, V3 b) { return V3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
  return V3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ V3 scale(V3 a, double s) { return V3{a.x * s, a.y * s, a.z * s}; }

// Closed-form int_T 1/R ds' and int_T (r' - rho)/R ds' (Wilton et al. 1984,
// Graglia 1993), rho = projection of r onto the plane of T.
__device__ void static_potentials(V3 r, V3 p0, V3 p1, V3 p2, double* Is, V3* Iv, V3* rho) {
  V3 n = cross(sub(p1, p0), sub(p2, p0));
  double nn = sqrt(dot(n, n));
  n = scale(n, 1.0 / nn);
  double h = dot(n, sub(r, p0));
  V3 rh = sub(r, scale(n, h));
  double ah = fabs(h);
  double s = 0.0;
  V3 v = V3{0.0, 0.0, 0.0};
  V3 P[3] = {p0, p1, p2};
  for (int e = 0; e < 3; ++e) {
    V3 pa = P[e], pb = P[(e + 1) % 3];
    V3 ed = sub(pb, pa);
    double elen = sqrt(dot(ed, ed));
    V3 lh = scale(ed, 1.0 / elen);
    V3 uh = cross(lh, n);
    double lp = dot(sub(pb, rh), lh);
    double lm = dot(sub(pa, rh), lh);
    double t = dot(sub(pa, rh), uh);
    double R0sq = t * t + h * h;
    double Rp = sqrt(R0sq + lp * lp);
    double Rm = sqrt(R0sq + lm * lm);
    bool degen = R0sq <= (1e-14 * elen) * (1e-14 * elen);
    double f = 0.0, beta = 0.0;
    if (!degen) {
      f = (lm + lp >= 0.0) ? log((Rp + lp) / (Rm + lm)) : log((Rm - lm) / (Rp - lp));
      if (ah > 0.0) beta = atan(t * lp / (R0sq + ah * Rp)) - atan(t * lm / (R0sq + ah * Rm));
    }
    s += t * f - ah * beta;
    double c = 0.5 * (R0sq * f + lp * Rp - lm * Rm);
    v.x += uh.x * c;
    v.y += uh.y * c;
    v.z += uh.z * c;
  }
  *Is = s;
  *Iv = v;
  *rho = rh;
}

// Pair sums of triangles a (test) and b (source): S[0] = S0, S[1..3] = S1,
// S[4..6] = S2, S[7] = S3.
__device__ void pair_moments(const MeshDev& M, int a, int b, double2 S[8]) {
  const int* ta = M.T + 3 * a;
  const int* tb = M.T + 3 * b;
  bool touch = false;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) touch |= (ta[i] == tb[j]);
  for (int i = 0; i < 8; ++i) S[i] = make_double2(0.0, 0.0);
  const double inv4pi = 1.0 / (4.0 * 3.141592653589793);
  const double k = M.k;
  for (int p = 0; p < 7; ++p) {
    V3 rp = v3(M.Q + (size_t)(7 * a + p) * 3);
    double2 gp = make_double2(0.0, 0.0);      // sum over q of w_q G
    double2 g1[3] = {{0, 0}, {0, 0}, {0, 0}};   // sum w_q G r_q
    double2 g3 = make_double2(0.0, 0.0);      // sum w_q G (r_p . r_q)
    for (int q = 0; q < 7; ++q) {
      V3 rq = v3(M.Q + (size_t)(7 * b + q) * 3);
      V3 d = sub(rp, rq);
      double R = sqrt(dot(d, d));
      double gr, gi;
      if (R == 0.0) {
        gr = 0.0;
        gi = -k * inv4pi;
      } else {
        double sn, cs;
        sincos(k * R, &sn, &cs);
        double ir = inv4pi / R;
        gr = (touch ? cs - 1.0 : cs) * ir;
        gi = -sn * ir;
      }
      double w = qw(q);
      gr *= w;
      gi *= w;
      gp.x += gr; gp.y += gi;
      g1[0].x += gr * rq.x; g1[0].y += gi * rq.x;
      g1[1].x += gr * rq.y; g1[1].y += gi * rq.y;
      g1[2].x += gr * rq.z; g1[2].y += gi * rq.z;
      double pq = dot(rp, rq);
      g3.x += gr * pq; g3.y += gi * pq;
    }
    double w = qw(p);
    S[0].x += w * gp.x; S[0].y += w * gp.y;
    for (int c = 0; c < 3; ++c) {
      S[1 + c].x += w * g1[c].x; S[1 + c].y += w * g1[c].y;
    }
    double rpc[3] = {rp.x, rp.y, rp.z};
    for (int c = 0; c < 3; ++c) {
      S[4 + c].x += w * gp.x * rpc[c]; S[4 + c].y += w * gp.y * rpc[c];
    }
    S[7].x += w * g3.x; S[7].y += w * g3.y;
  }
  if (touch) {
    int lo = min(a, b), hi = max(a, b);
    const int* th = M.T + 3 * hi;
    V3 p0 = v3(M.V + 3 * th[0]), p1 = v3(M.V + 3 * th[1]), p2 = v3(M.V + 3 * th[2]);
    double s0 = 0.0, s3 = 0.0;
    V3 sin_ = V3{0, 0, 0}, sout = V3{0, 0, 0};
    double sc0 = inv4pi / M.area[hi];
    for (int p = 0; p < 7; ++p) {
      V3 ro = v3(M.Q + (size_t)(7 * lo + p) * 3);
      double Is;
      V3 Iv, rh;
      static_potentials(ro, p0, p1, p2, &Is, &Iv, &rh);
      V3 Jv = V3{Iv.x + rh.x * Is, Iv.y + rh.y * Is, Iv.z + rh.z * Is};
      double sc = qw(p) * sc0;
      s0 += sc * Is;
      sin_.x += sc * Jv.x; sin_.y += sc * Jv.y; sin_.z += sc * Jv.z;
      sout.x += sc * Is * ro.x; sout.y += sc * Is * ro.y; sout.z += sc * Is * ro.z;
      s3 += sc * dot(ro, Jv);
    }
    if (a == b) {
      V3 mean = V3{0.5 * (sin_.x + sout.x), 0.5 * (sin_.y + sout.y), 0.5 * (sin_.z + sout.z)};
      sin_ = mean;
      sout = mean;
    }
    V3 m1 = (a > b) ? sout : sin_;
    V3 m2 = (a > b) ? sin_ : sout;
    S[0].x += s0;
    S[7].x += s3;
    S[1].x += m1.x; S[2].x += m1.y; S[3].x += m1.z;
    S[4].x += m2.x; S[5].x += m2.y; S[6].x += m2.z;
  }
}

// Z_mn for RWG indices m (test) and n (source).
__device__ double2 efie_entry(const MeshDev& M, int m, int n) {
  double2 t[2][2];
  for (int sa = 0; sa < 2; ++sa) {
    int a = M.tri[sa][m];
    V3 va = v3(M.V + 3 * M.T[3 * a + M.fv[sa][m]]);
    for (int sb = 0; sb < 2; ++sb) {
      int b = M.tri[sb][n];
      V3 vb = v3(M.V + 3 * M.T[3 * b + M.fv[sb][n]]);
      double2 S[8];
      pair_moments(M, a, b, S);
      double2 s2v = make_double2(S[4].x * vb.x + S[5].x * vb.y + S[6].x * vb.z,
                                 S[4].y * vb.x + S[5].y * vb.y + S[6].y * vb.z);
      double2 vs1 = make_double2(va.x * S[1].x + va.y * S[2].x + va.z * S[3].x,
                                 va.x * S[1].y + va.y * S[2].y + va.z * S[3].y);
      double vv = dot(va, vb);
      double2 A = make_double2(S[7].x - (s2v.x + vs1.x) + vv * S[0].x,
                               S[7].y - (s2v.y + vs1.y) + vv * S[0].y);
      double sg = (sa == sb) ? 1.0 : -1.0;
      double ll = M.len[m] * M.len[n] * sg;
      t[sa][sb] = make_double2(ll * ((M.k / 4.0) * A.x - S[0].x / M.k),
                               ll * ((M.k / 4.0) * A.y - S[0].y / M.k));
    }
  }
  double2 z = make_double2((t[0][0].x + t[1][1].x) + (t[0][1].x + t[1][0].x),
                           (t[0][0].y + t[1][1].y) + (t[0][1].y + t[1][0].y));
  // multiply by j eta
  return make_double2(-M.eta * z.y, M.eta * z.x);
}

}  // namespace hm
