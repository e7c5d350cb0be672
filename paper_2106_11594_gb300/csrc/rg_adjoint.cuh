// rg_adjoint.cuh -- gradient of a loss through the minimum-norm least-squares solution
// X = A^+ y, from the final factorization of a stream.
//
// With g = dL/dX, h = A^+T g, rho = y - A X, z = A^+T X and g_perp = (I - A^+ A) g, the
// derivative of the pseudoinverse on the manifold of matrices of fixed rank (obtained from
// the Penrose equations, Section 1) gives
//   dL/dy = h,   dL/dA = -h X^T + rho (A^+ h)^T + z g_perp^T.
// The factorization supplies A^+ = D^T P^-1 B^T (Section 2.1) with D the dual basis Ct
// (general variant) or Q (orthonormal variant), B = A D^T and P = B^T B; the row-space
// projector is A^+ A = D^T C. So, with the Cholesky factor of P already used for X:
//   a = D g, c = D X, e = C g,  alpha = P^-1 a,  beta = P^-1 c,
//   per row i: b = A_i D^T, h_i = b . alpha, z_i = b . beta, rho_i = y_i - A_i X,
//   B^T h = D (A^T h),  delta = P^-1 B^T h,  A^+ h = D^T delta,  g_perp = g - D^T e,
// and dL/dA is one elementwise pass over n x m. Everything is FP64.
#pragma once

#include "rg_core.cuh"

namespace rg {

struct AdjArgs {
  const double* A;  // n x m rows fed to the stream (row-major)
  const double* y;  // n
  long long n;
  const double* g;  // m: dL/dX
  double* gA;       // n x m
  double* gy;       // n
  double* X;        // m (scratch or caller's)
  double* Aph;      // m: A^+ h
  double* gperp;    // m
  double* v;        // m: A^T h
  double* a;        // r_max each: a, c, e, alpha, beta, B^T h, delta
  double* c;
  double* e;
  double* al;
  double* be;
  double* bth;
  double* de;
  double* h;    // n
  double* z;    // n
  double* rho;  // n
  double* part;  // row chunks x m partial sums of A^T h (grid teams), or null
  int nrc;       // row chunks of part
};

// r dot products D_k . x (warp per basis row), dealt over the team.
template <class Team>
__device__ void adj_rows_dot(const Team& T, const double* D, int ld, int m, int r, const double* x,
                             double* out) {
  const int lane = threadIdx.x & 31;
  const long long wstride = (long long)T.size() * NWARP;
  for (long long k = rr_warp(T); k < r; k += wstride) {
    const double* dk = D + (size_t)k * ld;
    double s = 0.0;
    for (int col = lane; col < m; col += 32) s = fma(__ldcg(dk + col), __ldcg(x + col), s);
    s = warp_sum(s);
    if (lane == 0) out[k] = s;
  }
}

// out[c] = base[c] + sign * sum_k D[k][c] x[k] over the team's threads (columns).
template <class Team>
__device__ void adj_cols(const Team& T, const double* D, int ld, int m, int r, const double* x,
                         const double* base, double sign, double* out) {
  const long long tstride = (long long)T.size() * NT;
  for (long long col = (long long)T.id() * NT + threadIdx.x; col < m; col += tstride) {
    double s = 0.0;
    for (int k = 0; k < r; ++k) s = fma(__ldcg(D + (size_t)k * ld + col), __ldcg(x + k), s);
    out[col] = (base ? __ldcg(base + col) : 0.0) + sign * s;
  }
}

// The whole adjoint for one stream, team-wide. Requires w formed and Lw = chol(P) for the
// current P (form_w). Returns false if a team barrier gave up.
template <class Team>
__device__ bool adjoint_run(const Team& T, const StreamDev& S, const AdjArgs& J, int r) {
  const int m = S.m, ld = S.ld, rm = S.r_max;
  const double* D = S.ortho ? S.C : S.Ct;
  const double* Cb = S.C;
  const long long n = J.n;
  const int lane = threadIdx.x & 31;
  // 1. X = D^T w
  adj_cols(T, D, ld, m, r, S.w, nullptr, 1.0, J.X);
  if (!T.sync()) return false;
  // 2. a = D g, c = D X, e = C g
  adj_rows_dot(T, D, ld, m, r, J.g, J.a);
  adj_rows_dot(T, D, ld, m, r, J.X, J.c);
  adj_rows_dot(T, Cb, ld, m, r, J.g, J.e);
  if (!T.sync()) return false;
  // 3. alpha = P^-1 a, beta = P^-1 c (worker 0)
  if (T.id() == 0 && r > 0) {
    cta_chol_solve(S.Lw, r, rm, J.a, J.al);
    cta_chol_solve(S.Lw, r, rm, J.c, J.be);
  }
  if (!T.sync()) return false;
  // 4. per row (one warp each): b = A_i D^T, h_i = b . alpha, z_i = b . beta, rho_i
  const long long wstride = (long long)T.size() * NWARP;
  for (long long i = rr_warp(T); i < n; i += wstride) {
    const double* ai = J.A + (size_t)i * m;
    double hz = 0.0, zz = 0.0;
    for (int k = 0; k < r; ++k) {
      const double* dk = D + (size_t)k * ld;
      double s = 0.0;
      for (int col = lane; col < m; col += 32) s = fma(__ldg(ai + col), __ldcg(dk + col), s);
      s = warp_sum(s);
      hz = fma(s, __ldcg(J.al + k), hz);
      zz = fma(s, __ldcg(J.be + k), zz);
    }
    double ax = 0.0;
    for (int col = lane; col < m; col += 32) ax = fma(__ldg(ai + col), __ldcg(J.X + col), ax);
    ax = warp_sum(ax);
    if (lane == 0) {
      J.h[i] = hz;
      J.z[i] = zz;
      J.rho[i] = __ldg(J.y + i) - ax;
    }
  }
  if (!T.sync()) return false;
  // 5. v = A^T h: row chunks x columns (fixed summation order)
  if (J.part) {
    const long long rows_per = (n + J.nrc - 1) / J.nrc;
    const long long items = (long long)J.nrc * ((m + NT - 1) / NT);
    for (long long it = T.id(); it < items; it += T.size()) {
      const int rc = (int)(it % J.nrc);
      const long long col = (it / J.nrc) * NT + threadIdx.x;
      if (col < m) {
        double s = 0.0;
        const long long i1 = min(n, (rc + 1) * rows_per);
        for (long long i = rc * rows_per; i < i1; ++i) s = fma(__ldcg(J.h + i), __ldg(J.A + (size_t)i * m + col), s);
        J.part[(size_t)rc * m + col] = s;
      }
    }
    if (!T.sync()) return false;
    const long long tstride = (long long)T.size() * NT;
    for (long long col = (long long)T.id() * NT + threadIdx.x; col < m; col += tstride) {
      double s = 0.0;
      for (int rc = 0; rc < J.nrc; ++rc) s += __ldcg(J.part + (size_t)rc * m + col);
      J.v[col] = s;
    }
  } else {
    for (long long col = threadIdx.x; col < m; col += NT) {
      double s = 0.0;
      for (long long i = 0; i < n; ++i) s = fma(__ldcg(J.h + i), __ldg(J.A + (size_t)i * m + col), s);
      J.v[col] = s;
    }
  }
  if (!T.sync()) return false;
  // 6. B^T h = D v; delta = P^-1 B^T h
  adj_rows_dot(T, D, ld, m, r, J.v, J.bth);
  if (!T.sync()) return false;
  if (T.id() == 0 && r > 0) cta_chol_solve(S.Lw, r, rm, J.bth, J.de);
  if (!T.sync()) return false;
  // 7. A^+ h = D^T delta, g_perp = g - D^T e
  adj_cols(T, D, ld, m, r, J.de, nullptr, 1.0, J.Aph);
  adj_cols(T, D, ld, m, r, J.e, J.g, -1.0, J.gperp);
  if (!T.sync()) return false;
  // 8. dL/dA = -h X^T + rho (A^+ h)^T + z g_perp^T, dL/dy = h
  const long long tstride = (long long)T.size() * NT;
  const long long nm = n * (long long)m;
  for (long long e2 = (long long)T.id() * NT + threadIdx.x; e2 < nm; e2 += tstride) {
    const long long i = e2 / m, col = e2 - i * m;
    const double v2 = -__ldcg(J.h + i) * __ldcg(J.X + col) + __ldcg(J.rho + i) * __ldcg(J.Aph + col) +
                      __ldcg(J.z + i) * __ldcg(J.gperp + col);
    J.gA[e2] = v2;
  }
  for (long long i = (long long)T.id() * NT + threadIdx.x; i < n; i += tstride) J.gy[i] = __ldcg(J.h + i);
  return true;
}

}  // namespace rg
