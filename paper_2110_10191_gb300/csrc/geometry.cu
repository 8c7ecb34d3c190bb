// geometry.cu -- device construction of the metric data of a simulation.
//
// The paper evaluates every metric-dependent quantity numerically from the
// analytic line element ("Implementation Notes", second paragraph): here
// g_{mu nu}(X) is evaluated in closed form, g^{mu nu} by a 4x4 inverse
// (adjugate / determinant), sqrt(-g) from the determinant, the lapse from
// g^{tt}, and the connection
//   Gamma^l_{mn} = 1/2 g^{lk} (d_m g_{kn} + d_n g_{km} - d_k g_{mn})
// with d_m by centred differences of step 1e-5 in X (d_t = 0: stationary).
// Both supported metrics are X3-independent, so one thread builds one (i,j)
// column and every location of it.
#include "grmhd_dev.cuh"
#include "grmhd_impl.h"

namespace grmhd {

constexpr double CONN_H = 1.0e-5;
constexpr double PI = 3.14159265358979323846;

__host__ __device__ void metric_at(int kind, double a, double h, double X1, double X2, double g[4][4]) {
#pragma unroll
  for (int m = 0; m < 4; m++)
#pragma unroll
    for (int n = 0; n < 4; n++) g[m][n] = 0.0;
  if (kind == 0) {
    g[0][0] = -1.0;
    g[1][1] = g[2][2] = g[3][3] = 1.0;
    return;
  }
  // Kerr (M = 1, spin a) in Kerr-Schild (t, r, theta, phi), then the diagonal
  // Jacobian to (t, X1, X2, X3): dr/dX1 = r, dtheta/dX2 = pi (1 + (1-h) cos 2 pi X2).
  const double r = exp(X1);
  const double th = PI * X2 + 0.5 * (1.0 - h) * sin(2.0 * PI * X2);
  double sth = sin(th);
  const double cth = cos(th);
  if (fabs(sth) < 1e-20) sth = (sth >= 0.0) ? 1e-20 : -1e-20;
  const double s2 = sth * sth;
  const double sig = r * r + a * a * cth * cth;
  const double tr = 2.0 * r / sig;  // 2 r / Sigma
  const double J1 = r;
  const double J2 = PI * (1.0 + (1.0 - h) * cos(2.0 * PI * X2));
  g[0][0] = -(1.0 - tr);
  g[0][1] = g[1][0] = tr * J1;
  g[0][3] = g[3][0] = -a * tr * s2;
  g[1][1] = (1.0 + tr) * J1 * J1;
  g[1][3] = g[3][1] = -a * s2 * (1.0 + tr) * J1;
  g[2][2] = sig * J2 * J2;
  g[3][3] = s2 * (sig + a * a * s2 * (1.0 + tr));
}

// inverse of a symmetric 4x4 by cofactors; returns the determinant
__host__ __device__ double inverse4(const double m[4][4], double inv[4][4]) {
  // 2x2 minors of the lower two rows and the upper two rows
  const double s0 = m[0][0] * m[1][1] - m[1][0] * m[0][1];
  const double s1 = m[0][0] * m[1][2] - m[1][0] * m[0][2];
  const double s2 = m[0][0] * m[1][3] - m[1][0] * m[0][3];
  const double s3 = m[0][1] * m[1][2] - m[1][1] * m[0][2];
  const double s4 = m[0][1] * m[1][3] - m[1][1] * m[0][3];
  const double s5 = m[0][2] * m[1][3] - m[1][2] * m[0][3];
  const double c5 = m[2][2] * m[3][3] - m[3][2] * m[2][3];
  const double c4 = m[2][1] * m[3][3] - m[3][1] * m[2][3];
  const double c3 = m[2][1] * m[3][2] - m[3][1] * m[2][2];
  const double c2 = m[2][0] * m[3][3] - m[3][0] * m[2][3];
  const double c1 = m[2][0] * m[3][2] - m[3][0] * m[2][2];
  const double c0 = m[2][0] * m[3][1] - m[3][0] * m[2][1];
  const double det = s0 * c5 - s1 * c4 + s2 * c3 + s3 * c2 - s4 * c1 + s5 * c0;
  const double id = 1.0 / det;
  inv[0][0] = (m[1][1] * c5 - m[1][2] * c4 + m[1][3] * c3) * id;
  inv[0][1] = (-m[0][1] * c5 + m[0][2] * c4 - m[0][3] * c3) * id;
  inv[0][2] = (m[3][1] * s5 - m[3][2] * s4 + m[3][3] * s3) * id;
  inv[0][3] = (-m[2][1] * s5 + m[2][2] * s4 - m[2][3] * s3) * id;
  inv[1][0] = (-m[1][0] * c5 + m[1][2] * c2 - m[1][3] * c1) * id;
  inv[1][1] = (m[0][0] * c5 - m[0][2] * c2 + m[0][3] * c1) * id;
  inv[1][2] = (-m[3][0] * s5 + m[3][2] * s2 - m[3][3] * s1) * id;
  inv[1][3] = (m[2][0] * s5 - m[2][2] * s2 + m[2][3] * s1) * id;
  inv[2][0] = (m[1][0] * c4 - m[1][1] * c2 + m[1][3] * c0) * id;
  inv[2][1] = (-m[0][0] * c4 + m[0][1] * c2 - m[0][3] * c0) * id;
  inv[2][2] = (m[3][0] * s4 - m[3][1] * s2 + m[3][3] * s0) * id;
  inv[2][3] = (-m[2][0] * s4 + m[2][1] * s2 - m[2][3] * s0) * id;
  inv[3][0] = (-m[1][0] * c3 + m[1][1] * c1 - m[1][2] * c0) * id;
  inv[3][1] = (m[0][0] * c3 - m[0][1] * c1 + m[0][2] * c0) * id;
  inv[3][2] = (-m[3][0] * s3 + m[3][1] * s1 - m[3][2] * s0) * id;
  inv[3][3] = (m[2][0] * s3 - m[2][1] * s1 + m[2][2] * s0) * id;
  return det;
}

__global__ void k_geometry(GeomArgs A) {
  const long long n2d = A.D.n2d;
  const long long ij = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (ij >= n2d) return;
  const int i = (int)(ij % A.D.s[0]);
  const int j = (int)(ij / A.D.s[0]);
  // global zone indices (a block of a decomposed grid sits at A.off)
  const int ig = i - NG + A.off[0], jg = j - NG + A.off[1];
  const double X1c = A.xmin[0] + (ig + 0.5) * A.dx[0];
  const double X2c = A.xmin[1] + (jg + 0.5) * A.dx[1];
  for (int loc = 0; loc < NLOC; loc++) {
    const double X1 = (loc == LOC_FACE1) ? A.xmin[0] + ig * A.dx[0] : X1c;
    const double X2 = (loc == LOC_FACE2) ? A.xmin[1] + jg * A.dx[1] : X2c;
    double g[4][4], gi[4][4];
    metric_at(A.kind, A.a, A.h, X1, X2, g);
    const double det = inverse4(g, gi);
    double *out = A.geom + (long long)loc * G_NCOMP * n2d;
    for (int m = 0; m < 4; m++)
      for (int n = m; n < 4; n++) {
        out[(G_GCOV + SY(m, n)) * n2d + ij] = g[m][n];
        out[(G_GCON + SY(m, n)) * n2d + ij] = gi[m][n];
      }
    const double gd = sqrt(fabs(det)), al = 1.0 / sqrt(-gi[0][0]);
    out[G_GDET * n2d + ij] = gd;
    out[G_ALPHA * n2d + ij] = al;
    out[G_IALPHA * n2d + ij] = 1.0 / al;
    out[G_IGDET * n2d + ij] = 1.0 / gd;
    // 1 - alpha = (1 - alpha^2)/(1 + alpha) with alpha^2 = -1/g^{tt}: no cancellation
    out[G_OMALPHA * n2d + ij] = (1.0 + 1.0 / gi[0][0]) / (1.0 + al);
    if (loc != LOC_CENT) continue;
    // connection at the centre: derivatives along X1, X2 (X3: the metric does
    // not depend on it, so that derivative is exactly zero)
    double dg[3][4][4];  // dg[m-1][k][n] = d_m g_{kn}, m = 1, 2
    for (int m = 1; m <= 2; m++) {
      double gp[4][4], gm[4][4];
      metric_at(A.kind, A.a, A.h, X1 + (m == 1 ? CONN_H : 0.0), X2 + (m == 2 ? CONN_H : 0.0), gp);
      metric_at(A.kind, A.a, A.h, X1 - (m == 1 ? CONN_H : 0.0), X2 - (m == 2 ? CONN_H : 0.0), gm);
      for (int k = 0; k < 4; k++)
        for (int n = 0; n < 4; n++) dg[m - 1][k][n] = (gp[k][n] - gm[k][n]) / (2.0 * CONN_H);
    }
    for (int k = 0; k < 4; k++)
      for (int n = 0; n < 4; n++) dg[2][k][n] = 0.0;
    // dgm(m, k, n) = d_m g_{kn}, zero for m = 0 and m = 3
    auto dgm = [&](int m, int k, int n) -> double { return (m == 1 || m == 2) ? dg[m - 1][k][n] : 0.0; };
    for (int l = 0; l < 4; l++)
      for (int m = 0; m < 4; m++)
        for (int n = m; n < 4; n++) {
          double acc = 0.0;
          for (int k = 0; k < 4; k++) acc += gi[l][k] * (dgm(m, k, n) + dgm(n, k, m) - dgm(k, m, n));
          A.conn[(l * 10 + SY(m, n)) * n2d + ij] = 0.5 * acc;
        }
    if (A.kind == 1) {
      const double r = exp(X1);
      const double kk = 1.0 / (r * r * (1.0 + r / 10.0));
      A.floors[0 * n2d + ij] = FL_RHO_K * kk;
      A.floors[1 * n2d + ij] = FL_U_K * pow(kk, A.gam);
    } else {
      A.floors[0 * n2d + ij] = 0.0;
      A.floors[1 * n2d + ij] = 0.0;
    }
  }
}

void launch_geometry(const GeomArgs &A, cudaStream_t st) {
  const int bs = 128;
  const long long nb = (A.D.n2d + bs - 1) / bs;
  k_geometry<<<(unsigned)nb, bs, 0, st>>>(A);
}

}  // namespace grmhd
