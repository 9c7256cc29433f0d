/*
 * dg_host.cpp -- host side of the DG library: reference rules, basis tables,
 * mesh validation, edge list and geometry, device upload and the C ABI entry
 * points (include/dg.h).
 *
 * Quadrature here is computed by the Golub-Welsch method: the nodes of an
 * n-point Gauss rule for a Jacobi weight are the eigenvalues of the symmetric
 * tridiagonal Jacobi matrix of the orthonormal recurrence, and the weights are
 * mu_0 times the squared first components of the normalised eigenvectors.  The
 * small symmetric eigenproblem is solved with cyclic Jacobi rotations.
 *
 * The basis is the orthonormal Dubiner basis on the reference triangle
 * {(0,0),(1,0),(0,1)} (the paper's Eq. np asks for an orthonormal basis of
 * degree <= p; this library fixes the Dubiner one):
 *   phi_ab(r, s) = N_ab P_a(alpha) (1-s)^a P_b^{(2a+1,0)}(beta),
 *   alpha = 2r/(1-s) - 1, beta = 2s - 1, N_ab = sqrt(2 (2a+1) (a+b+1)),
 * with Jacobi polynomials in their standard normalisation (three-term
 * recurrence), ordered by total degree a+b and then by b.
 */
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <vector>

#include "dg_internal.h"

namespace {

thread_local std::string g_err;

dg_status fail(dg_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

dg_status cuda_fail(cudaError_t e, const char *what) {
  return fail(DG_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define DG_CUDA(call, what)                      \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

// ---------------------------------------------------------------------------
// Gauss rules by Golub-Welsch.  Host tables are computed in long double and
// rounded once to double, so they are correct to the last bit or so.
// ---------------------------------------------------------------------------
using real = long double;

// Eigen-decomposition of a small symmetric matrix A (n x n, row-major) by cyclic
// Jacobi rotations.  On return A's diagonal holds the eigenvalues and the
// columns of V the orthonormal eigenvectors.
void sym_eigen(int n, std::vector<real> &A, std::vector<real> &V) {
  V.assign(n * n, 0.0L);
  for (int i = 0; i < n; ++i) V[i * n + i] = 1.0L;
  const real eps = std::numeric_limits<real>::epsilon();
  for (int sweep = 0; sweep < 100; ++sweep) {
    real off = 0.0L, diag = 0.0L;
    for (int i = 0; i < n; ++i) {
      diag += A[i * n + i] * A[i * n + i];
      for (int j = i + 1; j < n; ++j) off += A[i * n + j] * A[i * n + j];
    }
    if (off <= eps * eps * 1e-4L * (diag + 1e-300L)) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        real apq = A[p * n + q];
        if (apq == 0.0L) continue;
        real theta = (A[q * n + q] - A[p * n + p]) / (2.0L * apq);
        real t = (theta >= 0 ? 1.0L : -1.0L) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0L));
        real c = 1.0L / std::sqrt(t * t + 1.0L), s = t * c;
        for (int k = 0; k < n; ++k) {          // A <- A R  (columns p, q)
          real akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {          // A <- R^T A (rows p, q)
          real apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {          // V <- V R
          real vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
}

// n-point Gauss rule for the weight (1-x)^a (1+x)^b on [-1, 1], ascending nodes.
void gauss_rule(int n, real a, real b, std::vector<real> &x, std::vector<real> &w) {
  std::vector<real> J(n * n, 0.0L), V;
  for (int k = 0; k < n; ++k) {
    real s = 2.0L * k + a + b;
    J[k * n + k] = (k == 0) ? (b - a) / (a + b + 2.0L) : (b * b - a * a) / (s * (s + 2.0L));
    if (k >= 1) {
      real kk = k;
      real num = 4.0L * kk * (kk + a) * (kk + b) * (kk + a + b);
      real den = s * s * (s + 1.0L) * (s - 1.0L);
      real off = std::sqrt(num / den);
      J[(k - 1) * n + k] = off;
      J[k * n + (k - 1)] = off;
    }
  }
  sym_eigen(n, J, V);
  real mu0 = std::pow(2.0L, a + b + 1.0L) * std::exp(std::lgamma(a + 1.0L) + std::lgamma(b + 1.0L) -
                                                       std::lgamma(a + b + 2.0L));
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int i, int j) { return J[i * n + i] < J[j * n + j]; });
  x.resize(n);
  w.resize(n);
  for (int t = 0; t < n; ++t) {
    int i = idx[t];
    x[t] = J[i * n + i];
    w[t] = mu0 * V[0 * n + i] * V[0 * n + i];
  }
}

// Collapsed rule on the reference triangle: Gauss-Legendre in alpha, Gauss-Jacobi
// (1,0) in beta; r = (1+alpha)(1-beta)/4, s = (1+beta)/2, weight wa*wb/8.
// Point index = ib*n + ia.  The 1D nodes are rounded to double (xa, xb hold the
// rounded values); the points r, s are the exact images of the rounded nodes
// (extended precision), where every volume table is evaluated, and are stored
// rounded to double.
void collapsed_rule(int n, std::vector<real> &r, std::vector<real> &s, std::vector<real> &w,
                    std::vector<real> *xa_out = nullptr, std::vector<real> *xb_out = nullptr,
                    std::vector<real> *wa_out = nullptr, std::vector<real> *wb_out = nullptr) {
  std::vector<real> xa, wa, xb, wb;
  gauss_rule(n, 0.0L, 0.0L, xa, wa);
  gauss_rule(n, 1.0L, 0.0L, xb, wb);
  for (auto &v : xa) v = (real)(double)v;
  for (auto &v : xb) v = (real)(double)v;
  r.resize(n * n); s.resize(n * n); w.resize(n * n);
  for (int ib = 0; ib < n; ++ib)
    for (int ia = 0; ia < n; ++ia) {
      int k = ib * n + ia;
      r[k] = 0.25L * (1.0L + xa[ia]) * (1.0L - xb[ib]);
      s[k] = 0.5L * (1.0L + xb[ib]);
      w[k] = 0.125L * wa[ia] * wb[ib];
    }
  if (xa_out) *xa_out = xa;
  if (xb_out) *xb_out = xb;
  if (wa_out) *wa_out = wa;
  if (wb_out) *wb_out = wb;
}

// ---------------------------------------------------------------------------
// Dubiner basis from Jacobi recurrences
// ---------------------------------------------------------------------------

real jacobi_p(int n, real a, real b, real x) {
  if (n == 0) return 1.0L;
  real pm = 1.0L, pc = 0.5L * (a - b + (a + b + 2.0L) * x);
  for (int k = 1; k < n; ++k) {
    // P_{k+1} from P_k, P_{k-1}
    real kk = k;
    real s = 2.0L * kk + a + b;
    real A = 2.0L * (kk + 1.0L) * (kk + a + b + 1.0L) * s;
    real B = (s + 1.0L) * (a * a - b * b);
    real C = s * (s + 1.0L) * (s + 2.0L);
    real D = 2.0L * (kk + a) * (kk + b) * (s + 2.0L);
    real pn = ((B + C * x) * pc - D * pm) / A;
    pm = pc;
    pc = pn;
  }
  return pc;
}

real jacobi_dp(int n, real a, real b, real x) {
  if (n == 0) return 0.0L;
  return 0.5L * (n + a + b + 1.0L) * jacobi_p(n - 1, a + 1.0L, b + 1.0L, x);
}

void mode_ab(int j, int *a, int *b) {
  int k = 0;
  for (int d = 0;; ++d)
    for (int bb = 0; bb <= d; ++bb, ++k)
      if (k == j) { *a = d - bb; *b = bb; return; }
}

// phi_j and its reference gradient at (r, s) for every mode j of degree <= p
template <class T>
void dubiner_t(int p, real r, real s, T *phi, T *dr, T *ds) {
  int np = (p + 1) * (p + 2) / 2;
  real oms = 1.0L - s;
  real al = 2.0L * r / oms - 1.0L, be = 2.0L * s - 1.0L;
  for (int j = 0; j < np; ++j) {
    int a, b;
    mode_ab(j, &a, &b);
    real N = std::sqrt(2.0L * (2 * a + 1) * (a + b + 1));
    real Pa = jacobi_p(a, 0, 0, al), dPa = jacobi_dp(a, 0, 0, al);
    real Pb = jacobi_p(b, 2 * a + 1, 0, be), dPb = jacobi_dp(b, 2 * a + 1, 0, be);
    real oa = std::pow(oms, (real)a);
    real oa1 = a > 0 ? std::pow(oms, (real)(a - 1)) : 0.0L;
    if (phi) phi[j] = (T)(N * Pa * oa * Pb);
    // d/dr: d alpha/dr = 2/(1-s)
    if (dr) dr[j] = (T)(N * 2.0L * dPa * oa1 * Pb);
    // d/ds: d alpha/ds = (1+alpha)/(1-s), d beta/ds = 2
    if (ds) ds[j] = (T)(N * (oa1 * (dPa * (1.0L + al) - a * Pa) * Pb + 2.0L * Pa * oa * dPb));
  }
}

void dubiner(int p, real r, real s, double *phi, double *dr, double *ds) { dubiner_t<double>(p, r, s, phi, dr, ds); }

// ---------------------------------------------------------------------------
// Fully symmetric volume rules of degree 2p (Section 4.3.2 evaluates the volume
// integrals with rules of degree 2p; Section 6.1 gives their point counts, 3 at
// p = 1 and 16 at p = 4).  A rule invariant under the symmetries of the triangle is a
// union of orbits in barycentric coordinates, one weight per orbit:
//   S3    the centroid,                         1 point,  parameters (w)
//   S21   (a, a, 1-2a) and its permutations,    3 points, parameters (w, a)
//   S111  (a, b, 1-a-b) and its permutations,   6 points, parameters (w, a, b)
// (w is the weight of each point; (r, s) = the 2nd and 3rd barycentric
// coordinates).  The rule is exact to degree d when it integrates every
// orthonormal Dubiner polynomial of degree <= d exactly: sum_k w_k phi_j(x_k) =
// int phi_j = delta_j0 / sqrt(2).  The orbit structure for each p has as many
// parameters as there are independent symmetric conditions; they are solved by
// Gauss-Newton on all (2p+1)(2p+2)/2 conditions (normal equations, Gaussian
// elimination, extended precision, gradients from the basis derivatives) from
// the start values below.  Where several positive-interior rules of a structure
// exist (p = 3, p = 5), the start values pick the one whose points lie farthest
// from the edges.
// ---------------------------------------------------------------------------
struct SymOrbit {
  int kind;          // 0 = S3, 1 = S21, 2 = S111
  double prm[3];     // start values (w, a, b)
};
const SymOrbit kSym1[] = {{1, {0.167, 0.167}}};
const SymOrbit kSym2[] = {{1, {0.0550, 0.0916}}, {1, {0.112, 0.446}}};
const SymOrbit kSym3[] = {{1, {0.0254, 0.0631}}, {1, {0.0584, 0.249}}, {2, {0.0414, 0.0531, 0.310}}};
const SymOrbit kSym4[] = {{0, {0.0722}}, {1, {0.0162, 0.0505}}, {1, {0.0516, 0.171}}, {1, {0.0475, 0.459}},
                          {2, {0.0136, 0.00839, 0.263}}};
const SymOrbit kSym5[] = {{0, {0.0416}}, {1, {0.00548, 0.0285}}, {1, {0.0263, 0.163}},
                          {2, {0.0177, 0.0293, 0.363}}, {2, {0.0147, 0.0337, 0.153}},
                          {2, {0.0281, 0.147, 0.337}}};

struct SymPoint {
  real r, s, w;
  int iw, ia, ib;        // parameter indices of w, a, b (-1: none)
  real dra, drb, dsa, dsb;  // d r / d a, d r / d b, d s / d a, d s / d b
};

void sym_points(const SymOrbit *orb, int norb, const std::vector<real> &x, std::vector<SymPoint> &pts) {
  pts.clear();
  int off = 0;
  for (int o = 0; o < norb; ++o) {
    const real w = x[off];
    if (orb[o].kind == 0) {
      pts.push_back({1.0L / 3.0L, 1.0L / 3.0L, w, off, -1, -1, 0, 0, 0, 0});
      off += 1;
    } else if (orb[o].kind == 1) {
      const real a = x[off + 1], c = 1.0L - 2.0L * a;
      const int ia = off + 1;
      pts.push_back({a, a, w, off, ia, -1, 1, 0, 1, 0});
      pts.push_back({a, c, w, off, ia, -1, 1, 0, -2, 0});
      pts.push_back({c, a, w, off, ia, -1, -2, 0, 1, 0});
      off += 2;
    } else {
      const real a = x[off + 1], b = x[off + 2], c = 1.0L - a - b;
      const int ia = off + 1, ib = off + 2;
      // (value, d/da, d/db) of a, b, c
      const real v[3][3] = {{a, 1, 0}, {b, 0, 1}, {c, -1, -1}};
      const int order[6][2] = {{0, 1}, {1, 0}, {0, 2}, {2, 0}, {1, 2}, {2, 1}};
      for (auto &q : order)
        pts.push_back({v[q[0]][0], v[q[1]][0], w, off, ia, ib, v[q[0]][1], v[q[0]][2], v[q[1]][1], v[q[1]][2]});
      off += 3;
    }
  }
}

// solves A x = b in place (n x n, row-major; partial pivoting); false if singular
bool solve_dense(int n, std::vector<real> &A, std::vector<real> &b) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0L) return false;
    if (piv != c) {
      for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[piv * n + k]);
      std::swap(b[c], b[piv]);
    }
    for (int r = c + 1; r < n; ++r) {
      const real f = A[r * n + c] / A[c * n + c];
      for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
      b[r] -= f * b[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    real t = b[r];
    for (int k = r + 1; k < n; ++k) t -= A[r * n + k] * b[k];
    b[r] = t / A[r * n + r];
  }
  return true;
}

// The symmetric rule of degree 2p, rounded to double (r, s, w hold the rounded
// values).  false if p is unsupported or the iteration fails.
bool symmetric_rule(int p, std::vector<real> &r, std::vector<real> &s, std::vector<real> &w) {
  const SymOrbit *orb = nullptr;
  int norb = 0;
  switch (p) {
    case 1: orb = kSym1; norb = 1; break;
    case 2: orb = kSym2; norb = 2; break;
    case 3: orb = kSym3; norb = 3; break;
    case 4: orb = kSym4; norb = 5; break;
    case 5: orb = kSym5; norb = 6; break;
    default: return false;
  }
  std::vector<real> x;
  for (int o = 0; o < norb; ++o) {
    const int np_ = orb[o].kind == 0 ? 1 : orb[o].kind == 1 ? 2 : 3;
    for (int k = 0; k < np_; ++k) x.push_back((real)orb[o].prm[k]);
  }
  const int n = (int)x.size(), d = 2 * p, nm = (d + 1) * (d + 2) / 2;
  std::vector<SymPoint> pts;
  std::vector<real> phi(nm), dr(nm), ds(nm), res(nm), jac((size_t)nm * n);
  const real target0 = 1.0L / std::sqrt(2.0L);
  real worst = 0.0L;
  for (int it = 0; it < 60; ++it) {
    sym_points(orb, norb, x, pts);
    std::fill(res.begin(), res.end(), 0.0L);
    std::fill(jac.begin(), jac.end(), 0.0L);
    res[0] = -target0;
    for (const SymPoint &q : pts) {
      dubiner_t<real>(d, q.r, q.s, phi.data(), dr.data(), ds.data());
      for (int j = 0; j < nm; ++j) {
        res[j] += q.w * phi[j];
        real *g = &jac[(size_t)j * n];
        g[q.iw] += phi[j];
        if (q.ia >= 0) g[q.ia] += q.w * (dr[j] * q.dra + ds[j] * q.dsa);
        if (q.ib >= 0) g[q.ib] += q.w * (dr[j] * q.drb + ds[j] * q.dsb);
      }
    }
    worst = 0.0L;
    for (int j = 0; j < nm; ++j) worst = std::max(worst, std::fabs(res[j]));
    std::vector<real> A((size_t)n * n, 0.0L), b(n, 0.0L);
    for (int j = 0; j < nm; ++j) {
      const real *g = &jac[(size_t)j * n];
      for (int a = 0; a < n; ++a) {
        b[a] -= g[a] * res[j];
        for (int c = 0; c < n; ++c) A[a * n + c] += g[a] * g[c];
      }
    }
    if (!solve_dense(n, A, b)) return false;
    real step = 0.0L;
    for (int k = 0; k < n; ++k) {
      x[k] += b[k];
      step = std::max(step, std::fabs(b[k]));
    }
    if (step < std::max(64.0L * std::numeric_limits<real>::epsilon(), 1e-28L)) break;
  }
  if (!(worst < 1e-15L)) return false;
  sym_points(orb, norb, x, pts);
  r.resize(pts.size()); s.resize(pts.size()); w.resize(pts.size());
  for (size_t k = 0; k < pts.size(); ++k) {
    r[k] = (real)(double)pts[k].r;
    s[k] = (real)(double)pts[k].s;
    w[k] = (real)(double)pts[k].w;
    if (!(pts[k].w > 0.0L && pts[k].r > 0.0L && pts[k].s > 0.0L && pts[k].r + pts[k].s < 1.0L)) return false;
  }
  return true;
}

// The volume rule of a mesh: the collapsed grid or the symmetric rule.
bool volume_rule(int p, int rule, std::vector<real> &r, std::vector<real> &s, std::vector<real> &w) {
  if (rule == DG_RULE_COLLAPSED) {
    collapsed_rule(p + 1, r, s, w);
    return true;
  }
  if (rule == DG_RULE_SYMMETRIC) return symmetric_rule(p, r, s, w);
  return false;
}

// Reference point of edge coordinate xi on local face q (running from reference
// vertex q to vertex q+1).  The stored points are doubles: the node is rounded
// to double first and the point is formed in double arithmetic, and every basis
// table is evaluated (in extended precision) at exactly these double points.
void face_point(int q, real xi_, real *r, real *s) {
  static const double V[3][2] = {{0.0, 0.0}, {1.0, 0.0}, {0.0, 1.0}};
  const double xi = (double)xi_;
  int q1 = (q + 1) % 3;
  *r = (real)(0.5 * (1.0 - xi) * V[q][0] + 0.5 * (1.0 + xi) * V[q1][0]);
  *s = (real)(0.5 * (1.0 - xi) * V[q][1] + 0.5 * (1.0 + xi) * V[q1][1]);
}


bool supported(int p, int ne) {
  if (p < 1 || p > dg::PMAX) return false;
  return ne == p + 1 || (p == 3 && ne == 3);
}

void free_mesh(dg_mesh *m) {
  if (!m) return;
  cudaFree(m->geo); cudaFree(m->xy); cudaFree(m->elem_face); cudaFree(m->elem_nbr); cudaFree(m->face_conn);
  cudaFree(m->face_geo); cudaFree(m->table_block); cudaFree(m->trace); cudaFree(m->fhat);
  cudaFree(m->stage); cudaFree(m->host_state); cudaFree(m->rk_acc); cudaFree(m->partial); cudaFree(m->totals_dev);
  cudaFree(m->bstate); cudaFree(m->bxy);
  cudaFree(m->adj_buf);
  cudaFree(m->err_flag);
  cudaFree(m->gbar);
  cudaFree(m->tc_img[0]); cudaFree(m->tc_img[1]);
  if (m->copy_stream) cudaStreamDestroy(m->copy_stream);
  for (auto &e : m->copy_ev)
    if (e) cudaEventDestroy(e);
  if (m->timing) {
    for (auto &r : m->timing->pool) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    delete m->timing;
  }
  if (m->graph) {
    if (m->graph->exec) cudaGraphExecDestroy(m->graph->exec);
    if (m->graph->ready) cudaEventDestroy(m->graph->ready);
    if (m->graph->done) cudaEventDestroy(m->graph->done);
    if (m->graph->stream) cudaStreamDestroy(m->graph->stream);
    delete m->graph;
  }
  delete m;
}

// Runs one launcher; with timing on, brackets it with an event pair on `stream`.
template <class F>
int timed(dg_mesh *m, int kind, void *stream, F &&launch) {
  dg::Timing *t = m->timing;
  if (!t || !t->on) return launch();
  if (t->used == t->pool.size()) {
    dg::Timing::Rec r{};
    if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) {
      cudaGetLastError();
      return launch();
    }
    t->pool.push_back(r);
  }
  dg::Timing::Rec &r = t->pool[t->used];
  cudaEventRecord(r.a, (cudaStream_t)stream);
  int e = launch();
  cudaEventRecord(r.b, (cudaStream_t)stream);
  r.kind = kind;
  ++t->used;
  return e;
}

}  // namespace

namespace dg {
dg_status set_error(dg_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}
}  // namespace dg

// ===========================================================================
// C ABI
// ===========================================================================

extern "C" const char *dg_last_error(void) { return g_err.c_str(); }

// Kernels launch on the current device; the mesh's arrays live on the device it
// was created on.
static dg_status check_device(const dg_mesh *m, const char *who) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(DG_ECUDA, "%s: cudaGetDevice failed", who);
  }
  if (dev != m->device)
    return fail(DG_EINVAL, "%s: the current device is %d, the mesh lives on device %d", who, dev, m->device);
  return DG_OK;
}

extern "C" dg_status dg_host_tables(int p, int ne, double *vol_r, double *vol_s, double *vol_w,
                                    double *edge_x, double *edge_w, double *phi, double *dphi_r,
                                    double *dphi_s, double *phi_face) {
  if (ne == 0) ne = p + 1;
  if (p < 0 || p > 8 || ne < 1 || ne > 16) return fail(DG_EINVAL, "dg_host_tables: p=%d ne=%d", p, ne);
  int np = (p + 1) * (p + 2) / 2, nd = p + 1, nq = nd * nd;
  std::vector<real> r, s, w, ex, ew;
  collapsed_rule(nd, r, s, w);
  gauss_rule(ne, 0.0L, 0.0L, ex, ew);
  for (int k = 0; k < nq; ++k) {
    if (vol_r) vol_r[k] = (double)r[k];
    if (vol_s) vol_s[k] = (double)s[k];
    if (vol_w) vol_w[k] = (double)w[k];
    dubiner(p, r[k], s[k], phi ? phi + k * np : nullptr, dphi_r ? dphi_r + k * np : nullptr,
            dphi_s ? dphi_s + k * np : nullptr);
  }
  for (int k = 0; k < ne; ++k) {
    if (edge_x) edge_x[k] = (double)ex[k];
    if (edge_w) edge_w[k] = (double)ew[k];
  }
  if (phi_face)
    for (int q = 0; q < 3; ++q)
      for (int k = 0; k < ne; ++k) {
        real rr, ss;
        face_point(q, ex[k], &rr, &ss);
        dubiner(p, rr, ss, phi_face + (q * ne + k) * np, nullptr, nullptr);
      }
  g_err.clear();
  return DG_OK;
}

extern "C" dg_status dg_volume_rule(int p, int rule, int *nq, double *r, double *s, double *w, double *phi) {
  if (!nq || p < 1 || p > dg::PMAX) return fail(DG_EINVAL, "dg_volume_rule: p=%d", p);
  std::vector<real> vr, vs, vw;
  if (rule != DG_RULE_COLLAPSED && rule != DG_RULE_SYMMETRIC) return fail(DG_EINVAL, "dg_volume_rule: rule=%d", rule);
  if (!volume_rule(p, rule, vr, vs, vw)) return fail(DG_EINVAL, "dg_volume_rule: no rule for p=%d", p);
  const int n = (int)vr.size(), np = (p + 1) * (p + 2) / 2;
  *nq = n;
  for (int k = 0; k < n; ++k) {
    if (r) r[k] = (double)vr[k];
    if (s) s[k] = (double)vs[k];
    if (w) w[k] = (double)vw[k];
    if (phi) dubiner(p, vr[k], vs[k], phi + (size_t)k * np, nullptr, nullptr);
  }
  g_err.clear();
  return DG_OK;
}

extern "C" dg_status dg_mesh_create(const dg_mesh_desc *d, dg_mesh **out) {
  using namespace dg;
  if (!d || !out) return fail(DG_EINVAL, "dg_mesh_create: null argument");
  *out = nullptr;
  if (!d->elem_xy || !d->nbr || !d->nbr_face) return fail(DG_EINVAL, "dg_mesh_create: null mesh array");
  const int64_t N = d->n_elem;
  if (N < 1 || N > (int64_t)INT32_MAX / 3) return fail(DG_EINVAL, "dg_mesh_create: n_elem=%lld", (long long)N);
  const int p = d->p;
  const int ne = d->n_edge_pts ? d->n_edge_pts : p + 1;
  if (!supported(p, ne)) return fail(DG_EINVAL, "dg_mesh_create: unsupported p=%d n_edge_pts=%d", p, ne);
  if (!(d->gamma > 1.0)) return fail(DG_EINVAL, "dg_mesh_create: gamma must exceed 1");
  if (d->vol_rule != DG_RULE_COLLAPSED && d->vol_rule != DG_RULE_SYMMETRIC)
    return fail(DG_EINVAL, "dg_mesh_create: unknown vol_rule %d", d->vol_rule);

  const double *xy = d->elem_xy;
  // --- validation and edge list ------------------------------------------
  std::vector<double> geo(N * GEO);
  double rin_min = INFINITY;
  for (int64_t e = 0; e < N; ++e) {
    const double *v = xy + 6 * e;
    double a = v[2] - v[0], b = v[4] - v[0], c = v[3] - v[1], dd = v[5] - v[1];
    double det = a * dd - b * c;
    if (!(det > 0.0) || !std::isfinite(det))
      return fail(DG_EMESH, "element %lld is not counter-clockwise (det J = %g)", (long long)e, det);
    double *g = &geo[e * GEO];
    g[0] = dd; g[1] = -b; g[2] = -c; g[3] = a;      // det J * J^{-1}
    const double per = std::hypot(a, c) + std::hypot(b, dd) + std::hypot(b - a, dd - c);
    rin_min = std::min(rin_min, det / per);         // inscribed radius = 2 area / perimeter
    g[4] = 1.0 / det; g[5] = det; g[6] = 0.0; g[7] = 0.0;
  }
  std::vector<int32_t> elem_face(N * 3, -1);
  std::vector<FaceConn> conn;
  std::vector<FaceGeo> fgeo;
  conn.reserve(N * 3 / 2 + 1);
  fgeo.reserve(N * 3 / 2 + 1);
  auto face_geo = [&](const double *v, int q) {
    // l = |edge| / 2 (Eq. len); the flux is scaled by h = l / 2 (F_hat's 1/2)
    const int q1 = (q + 1) % 3;
    const double dx = v[2 * q1] - v[2 * q], dy = v[2 * q1 + 1] - v[2 * q + 1];
    const double len = std::sqrt(dx * dx + dy * dy);
    const double nx = dy / len, ny = -dx / len, l = 0.5 * len, h = 0.5 * l, g1 = d->gamma - 1.0;
    return FaceGeo{nx, ny, l, h * h * d->gamma * g1, h * nx, h * ny, g1 * (h * nx), g1 * (h * ny)};
  };
  // boundary faces first (as the paper sorts its edge list: the warps of the edge
  // kernels then take one branch), in element order; the element is the left side
  int64_t n_state = 0;
  for (int64_t e = 0; e < N; ++e)
    for (int q = 0; q < 3; ++q) {
      const int64_t f = d->nbr[3 * e + q];
      if (f >= 0) continue;
      if (f != DG_BC_WALL && f != DG_BC_STATE)
        return fail(DG_EMESH, "element %lld face %d: boundary code %lld is not DG_BC_WALL or DG_BC_STATE",
                    (long long)e, q, (long long)f);
      if (f == DG_BC_STATE) ++n_state;
      elem_face[3 * e + q] = 2 * (int32_t)conn.size();
      conn.push_back(FaceConn{(int32_t)e, q, (int32_t)f, -1});
      fgeo.push_back(face_geo(xy + 6 * e, q));
    }
  const int64_t Fb = (int64_t)conn.size();
  for (int64_t e = 0; e < N; ++e)
    for (int q = 0; q < 3; ++q) {
      int64_t f = d->nbr[3 * e + q];
      int qf = d->nbr_face[3 * e + q];
      if (f < 0) continue;
      if (f >= N || qf < 0 || qf > 2)
        return fail(DG_EMESH, "element %lld face %d: neighbour (%lld, %d) out of range", (long long)e, q,
                    (long long)f, qf);
      if (d->nbr[3 * f + qf] != e || d->nbr_face[3 * f + qf] != q)
        return fail(DG_EMESH, "element %lld face %d: neighbour relation is not symmetric", (long long)e, q);
      if (f == e && qf == q) return fail(DG_EMESH, "element %lld face %d is its own neighbour", (long long)e, q);
      const double *v = xy + 6 * e, *w = xy + 6 * f;
      int q1 = (q + 1) % 3, qf1 = (qf + 1) % 3;
      double dx = v[2 * q1] - v[2 * q], dy = v[2 * q1 + 1] - v[2 * q + 1];
      double len = std::sqrt(dx * dx + dy * dy);
      // the neighbour traverses the edge backwards: v_q ~ w_{qf+1}, v_{q+1} ~ w_qf
      double t0x = v[2 * q] - w[2 * qf1], t0y = v[2 * q + 1] - w[2 * qf1 + 1];
      double t1x = v[2 * q1] - w[2 * qf], t1y = v[2 * q1 + 1] - w[2 * qf + 1];
      if (std::fabs(t0x - t1x) > 1e-9 * len || std::fabs(t0y - t1y) > 1e-9 * len)
        return fail(DG_EMESH, "element %lld face %d: the neighbour's edge is not a translate", (long long)e, q);
      if (!(e < f || (e == f && q < qf))) continue;
      int32_t fi = (int32_t)conn.size();
      conn.push_back(FaceConn{(int32_t)e, q, (int32_t)f, qf});
      fgeo.push_back(face_geo(v, q));
      elem_face[3 * e + q] = 2 * fi + 0;
      elem_face[3 * f + qf] = 2 * fi + 1;
    }
  const int64_t F = (int64_t)conn.size();

  // --- tables ----------------------------------------------------------------
  const int np = (p + 1) * (p + 2) / 2, nd = p + 1, nf = 3 * ne;
  std::vector<real> r, s, w, ex, ew, xa, xb, wa_, wb_;
  // the collapsed grid's 1D rules feed the sum-factorisation tables whichever
  // volume rule the mesh uses (the edge tables need them too)
  collapsed_rule(nd, r, s, w, &xa, &xb, &wa_, &wb_);
  if (d->vol_rule == DG_RULE_SYMMETRIC && !symmetric_rule(p, r, s, w))
    return fail(DG_EINVAL, "dg_mesh_create: the symmetric rule for p=%d did not converge", p);
  const int nq = (int)r.size();
  gauss_rule(ne, 0.0L, 0.0L, ex, ew);
  std::vector<double> phi(nq * np), dr(nq * np), ds(nq * np), phif(nf * np);
  for (int k = 0; k < nq; ++k) dubiner(p, r[k], s[k], &phi[k * np], &dr[k * np], &ds[k * np]);
  for (int q = 0; q < 3; ++q)
    for (int k = 0; k < ne; ++k) {
      real rr, ss;
      face_point(q, ex[k], &rr, &ss);
      dubiner(p, rr, ss, &phif[(q * ne + k) * np], nullptr, nullptr);
    }
  size_t off = 0;
  auto take = [&](size_t n) { size_t o = off; off += (n + 3) & ~size_t(3); return o; };
  size_t oBvT = take(np * nq), oDr = take(nq * np), oDs = take(nq * np), oLf = take(nf * np),
         oBfT = take(np * nf), oPw = take(nq * np), oVr = take(nq), oVs = take(nq);
  size_t oSPa = take(nd * nd), oSPaW = take(nd * nd), oSdPaW = take(nd * nd), oSChi = take(np * nd),
         oSChiA = take(np * nd), oSdChiB = take(np * nd), oSHalf = take(nd);
  size_t oEChi = take(np * ne), oEWChi = take(np * ne), oEWPa = take(nd * ne), oEChiM1 = take(np),
         oEPa = take(nd * ne);
  std::vector<double> tb(off, 0.0);
  for (int k = 0; k < nq; ++k)
    for (int j = 0; j < np; ++j) {
      tb[oBvT + j * nq + k] = phi[k * np + j];
      tb[oDr + k * np + j] = (double)(w[k] * (real)dr[k * np + j]);
      tb[oDs + k * np + j] = (double)(w[k] * (real)ds[k * np + j]);
      tb[oPw + k * np + j] = (double)(w[k] * (real)phi[k * np + j]);
    }
  for (int q = 0; q < 3; ++q)
    for (int k = 0; k < ne; ++k)
      for (int j = 0; j < np; ++j) {
        int qk = q * ne + k;
        tb[oLf + qk * np + j] = (double)(ew[k] * (real)phif[qk * np + j]);
        tb[oBfT + j * nf + qk] = phif[qk * np + j];
      }
  for (int k = 0; k < nq; ++k) { tb[oVr + k] = (double)r[k]; tb[oVs + k] = (double)s[k]; }
  // sum-factorisation tables.  The volume weight w = wa(ia) wb(ib) / 8 and the
  // chain-rule factors of the collapsed map are folded into the projection
  // tables: the element kernel forms H_alpha = G_r + (1+alpha)/2 G_s and
  // H_beta = G_s at the points, and
  //   V_j = sum_ib chiA_j(ib) sum_ia wa P_a'(alpha_ia) H_alpha
  //       + sum_ib dchiB_j(ib) sum_ia wa P_a(alpha_ia) H_beta,
  //   chiA_j = chi_j wb / (4 (1-s)),  dchiB_j = chi_j' wb / 4,
  // which is the projection on w (d phi_j/dr, d phi_j/ds) . (G_r, G_s) with
  // d/dr = 2/(1-s) d/dalpha and d/ds = (1+alpha)/(1-s) d/dalpha + 2 d/dbeta.
  for (int a = 0; a < nd; ++a)
    for (int ia = 0; ia < nd; ++ia) {
      const real P = jacobi_p(a, 0, 0, xa[ia]), dP = jacobi_dp(a, 0, 0, xa[ia]);
      tb[oSPa + a * nd + ia] = (double)P;
      tb[oSPaW + a * nd + ia] = (double)(wa_[ia] * P);
      tb[oSdPaW + a * nd + ia] = (double)(wa_[ia] * dP);
    }
  for (int j = 0; j < np; ++j) {
    int a, b;
    mode_ab(j, &a, &b);
    real N = std::sqrt(2.0L * (2 * a + 1) * (a + b + 1));
    for (int ib = 0; ib < nd; ++ib) {
      real be = xb[ib], h = 0.5L * (1.0L - be);   // h = 1 - s
      real Pb = jacobi_p(b, 2 * a + 1, 0, be), dPb = jacobi_dp(b, 2 * a + 1, 0, be);
      real ha = std::pow(h, (real)a), ha1 = a > 0 ? std::pow(h, (real)(a - 1)) : 0.0L;
      const real chi = N * ha * Pb, dchi = N * (-0.5L * a * ha1 * Pb + ha * dPb);
      tb[oSChi + j * nd + ib] = (double)chi;
      tb[oSChiA + j * nd + ib] = (double)(chi * wb_[ib] / (4.0L * h));
      tb[oSdChiB + j * nd + ib] = (double)(dchi * wb_[ib] / 4.0L);
    }
  }
  for (int ia = 0; ia < nd; ++ia) tb[oSHalf + ia] = (double)(0.5L * (1.0L + xa[ia]));
  // sum-factorisation tables of the edges.  On the reference edges the collapsed
  // coordinates are: face 0 (v0 -> v1) alpha = xi, beta = -1; face 1 (v1 -> v2)
  // alpha = 1, beta = xi; face 2 (v2 -> v0) alpha = -1, beta = -xi.  With
  // P_a(1) = 1 and P_a(-1) = (-1)^a, the traces of faces 1 and 2 are
  //   T1_k = sum_a Y_a(xi_k),  T2_k = sum_a (-1)^a Y_a(xi_{ne-1-k}),
  //   Y_a(xi) = sum_b chi_ab(xi) c_ab
  // (the Gauss-Legendre nodes are symmetric, -xi_k = xi_{ne-1-k}), and the lift
  // is the transposed sum with the weights omega_k; on face 0 it is
  //   chi_j(-1) sum_k omega_k P_a(xi_k) F_k.
  for (int k = 0; k < ne; ++k) {
    const real x = (real)(double)ex[k];      // the edge points are formed from the rounded node
    for (int a = 0; a < nd; ++a) {
      tb[oEWPa + a * ne + k] = (double)(ew[k] * jacobi_p(a, 0, 0, x));
      tb[oEPa + a * ne + k] = (double)jacobi_p(a, 0, 0, x);
    }
  }
  for (int j = 0; j < np; ++j) {
    int a, b;
    mode_ab(j, &a, &b);
    const real N = std::sqrt(2.0L * (2 * a + 1) * (a + b + 1));
    for (int k = 0; k < ne; ++k) {
      const real x = (real)(double)ex[k];
      const real chi = N * std::pow(0.5L * (1.0L - x), (real)a) * jacobi_p(b, 2 * a + 1, 0, x);
      tb[oEChi + j * ne + k] = (double)chi;
      tb[oEWChi + j * ne + k] = (double)(ew[k] * chi);
    }
    tb[oEChiM1 + j] = (double)(N * jacobi_p(b, 2 * a + 1, 0, -1.0L));
  }

  // --- device upload ---------------------------------------------------------
  dg_mesh *m = new (std::nothrow) dg_mesh();
  if (!m) return fail(DG_ENOMEM, "dg_mesh_create: host allocation");
  m->timing = new (std::nothrow) dg::Timing();
  if (!m->timing) { delete m; return fail(DG_ENOMEM, "dg_mesh_create: host allocation"); }
  m->p = p; m->np = np; m->nq = nq; m->nd = nd; m->ne = ne; m->gamma = d->gamma; m->rule = d->vol_rule;
  m->N = N; m->F = F;
  m->rin_min = rin_min;
  m->phi1 = phi[0];                              // phi_1 at the first volume point: the constant mode
  cudaGetDevice(&m->device);
  if (cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, m->device) != cudaSuccess || m->num_sms < 1) {
    cudaGetLastError();
    m->num_sms = 1;
  }
  auto dalloc = [&](void **ptr, size_t bytes, const char *what) -> dg_status {
    cudaError_t e = cudaMalloc(ptr, bytes ? bytes : 16);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(DG_ENOMEM, "cudaMalloc(%s, %zu bytes): %s", what, bytes, cudaGetErrorString(e));
    }
    return DG_OK;
  };
  dg_status st;
#define DG_ALLOC(ptr, bytes, what) \
  if ((st = dalloc((void **)&(ptr), (bytes), (what))) != DG_OK) { free_mesh(m); return st; }
  DG_ALLOC(m->geo, sizeof(double) * N * GEO, "geometry");
  DG_ALLOC(m->xy, sizeof(double) * N * 6, "vertices");
  DG_ALLOC(m->elem_face, sizeof(int32_t) * N * 3, "element faces");
  DG_ALLOC(m->elem_nbr, sizeof(int32_t) * N * 3, "element neighbours");
  DG_ALLOC(m->face_conn, sizeof(FaceConn) * F, "face connectivity");
  DG_ALLOC(m->face_geo, sizeof(FaceGeo) * F, "face geometry");
  DG_ALLOC(m->table_block, sizeof(double) * off, "tables");
  DG_ALLOC(m->trace, sizeof(double) * N * nf * M, "traces");
  DG_ALLOC(m->fhat, sizeof(double) * F * ne * M, "edge fluxes");
  DG_ALLOC(m->stage, sizeof(double) * N * M * np, "stage buffer");
  m->totals_blocks = 256;
  DG_ALLOC(m->partial, sizeof(double) * m->totals_blocks * M, "totals partials");
  DG_ALLOC(m->totals_dev, sizeof(double) * M, "totals");
  DG_ALLOC(m->err_flag, sizeof(int), "error flag");
  DG_ALLOC(m->gbar, 2 * sizeof(unsigned), "grid barrier");
  m->small_stepper = 1;
  m->Fb = Fb;
  m->n_state_faces = n_state;
  m->bstate_set = n_state == 0;
  if (Fb > 0) {
    DG_ALLOC(m->bstate, sizeof(double) * Fb * ne * M, "boundary states");
    DG_ALLOC(m->bxy, sizeof(double) * Fb * ne * 2, "boundary points");
  }
#undef DG_ALLOC
  m->table_doubles = off;
  double *T = m->table_block;
  m->tab.BvT = T + oBvT; m->tab.Dr = T + oDr; m->tab.Ds = T + oDs; m->tab.Lf = T + oLf;
  m->tab.BfT = T + oBfT; m->tab.Pw = T + oPw; m->tab.vr = T + oVr; m->tab.vs = T + oVs;
  m->tab.SPa = T + oSPa; m->tab.SPaW = T + oSPaW; m->tab.SdPaW = T + oSdPaW; m->tab.SChi = T + oSChi;
  m->tab.SChiA = T + oSChiA; m->tab.SdChiB = T + oSdChiB; m->tab.SHalf = T + oSHalf;
  m->tab.EChi = T + oEChi; m->tab.EWChi = T + oEWChi; m->tab.EWPa = T + oEWPa;
  m->tab.EChiM1 = T + oEChiM1;
  m->tab.EPa = T + oEPa;
  // the neighbour across each face; a boundary face adds the element itself
  std::vector<int32_t> elem_nbr(N * 3);
  for (int64_t i = 0; i < N * 3; ++i) elem_nbr[i] = d->nbr[i] >= 0 ? (int32_t)d->nbr[i] : (int32_t)(i / 3);
  // physical points of the boundary faces (Eq. 1dmap at the edge nodes, in the
  // element's counter-clockwise direction)
  std::vector<double> bxy(Fb * ne * 2);
  for (int64_t b = 0; b < Fb; ++b) {
    const double *v = xy + 6 * conn[b].l;
    const int q = conn[b].L, q1 = (q + 1) % 3;
    for (int k = 0; k < ne; ++k) {
      const double t = (double)ex[k];
      bxy[(b * ne + k) * 2 + 0] = 0.5 * (1.0 - t) * v[2 * q] + 0.5 * (1.0 + t) * v[2 * q1];
      bxy[(b * ne + k) * 2 + 1] = 0.5 * (1.0 - t) * v[2 * q + 1] + 0.5 * (1.0 + t) * v[2 * q1 + 1];
    }
  }
  cudaError_t ce;
  if (Fb > 0 &&
      ((ce = cudaMemcpy(m->bxy, bxy.data(), sizeof(double) * Fb * ne * 2, cudaMemcpyHostToDevice)) != cudaSuccess ||
       (ce = cudaMemset(m->bstate, 0, sizeof(double) * Fb * ne * M)) != cudaSuccess)) {
    free_mesh(m);
    return cuda_fail(ce, "dg_mesh_create: boundary upload");
  }
  if ((ce = cudaMemcpy(m->geo, geo.data(), sizeof(double) * N * GEO, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (ce = cudaMemcpy(m->elem_nbr, elem_nbr.data(), sizeof(int32_t) * N * 3, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (ce = cudaMemcpy(m->xy, xy, sizeof(double) * N * 6, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (ce = cudaMemcpy(m->elem_face, elem_face.data(), sizeof(int32_t) * N * 3, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (ce = cudaMemcpy(m->face_conn, conn.data(), sizeof(FaceConn) * F, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (ce = cudaMemcpy(m->face_geo, fgeo.data(), sizeof(FaceGeo) * F, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (ce = cudaMemcpy(m->table_block, tb.data(), sizeof(double) * off, cudaMemcpyHostToDevice)) != cudaSuccess ||
      (ce = cudaMemset(m->err_flag, 0, sizeof(int))) != cudaSuccess ||
      (ce = (cudaError_t)dg::tc_tables(m)) != cudaSuccess) {
    free_mesh(m);
    return cuda_fail(ce, "dg_mesh_create: upload");
  }
  *out = m;
  g_err.clear();
  return DG_OK;
}

extern "C" dg_status dg_mesh_destroy(dg_mesh *m) {
  if (!m) return DG_OK;
  cudaDeviceSynchronize();
  free_mesh(m);
  return DG_OK;
}

extern "C" dg_status dg_mesh_info(const dg_mesh *m, dg_mesh_info_t *info) {
  if (!m || !info) return fail(DG_EINVAL, "dg_mesh_info: null argument");
  info->n_elem = m->N; info->n_face = m->F; info->p = m->p; info->n_modes = m->np;
  info->n_vol_pts = m->nq; info->n_edge_pts = m->ne; info->gamma = m->gamma;
  info->n_boundary_face = m->Fb;
  return DG_OK;
}

extern "C" dg_status dg_boundary_points(const dg_mesh *m, double *xy, void *stream) {
  if (!m || !xy) return fail(DG_EINVAL, "dg_boundary_points: null argument");
  if (dg_status dst = check_device(m, "dg_boundary_points")) return dst;
  if (m->Fb == 0) return DG_OK;
  DG_CUDA(cudaMemcpyAsync(xy, m->bxy, sizeof(double) * m->Fb * m->ne * 2, cudaMemcpyDeviceToDevice,
                          (cudaStream_t)stream), "dg_boundary_points");
  return DG_OK;
}

extern "C" dg_status dg_set_boundary_state(dg_mesh *m, const double *u, void *stream) {
  if (!m || !u) return fail(DG_EINVAL, "dg_set_boundary_state: null argument");
  if (dg_status dst = check_device(m, "dg_set_boundary_state")) return dst;
  if (m->Fb == 0) return DG_OK;
  DG_CUDA(cudaMemcpyAsync(m->bstate, u, sizeof(double) * m->Fb * m->ne * dg::M, cudaMemcpyDeviceToDevice,
                          (cudaStream_t)stream), "dg_set_boundary_state");
  m->bstate_set = true;
  return DG_OK;
}

extern "C" dg_status dg_volume_points(const dg_mesh *m, double *xy, void *stream) {
  if (!m || !xy) return fail(DG_EINVAL, "dg_volume_points: null argument");
  if (dg_status dst = check_device(m, "dg_volume_points")) return dst;
  DG_CUDA((cudaError_t)dg::launch_volume_points(m, xy, stream), "dg_volume_points");
  return DG_OK;
}

extern "C" dg_status dg_eval_points(dg_mesh *m, int npts, const double *r, const double *s, const double *c,
                                    double *out, void *stream) {
  if (!m || !r || !s || !c || !out) return fail(DG_EINVAL, "dg_eval_points: null argument");
  if (dg_status dst = check_device(m, "dg_eval_points")) return dst;
  if (npts < 1 || npts > 1 << 20) return fail(DG_EINVAL, "dg_eval_points: npts=%d", npts);
  std::vector<double> tab((size_t)npts * m->np);
  for (int k = 0; k < npts; ++k) {
    if (!(r[k] >= 0.0 && s[k] >= 0.0 && r[k] + s[k] < 1.0))
      return fail(DG_EINVAL, "dg_eval_points: point %d = (%g, %g) is not inside the reference triangle", k, r[k], s[k]);
    dubiner(m->p, (real)r[k], (real)s[k], &tab[(size_t)k * m->np], nullptr, nullptr);
  }
  double *dtab = nullptr;
  DG_CUDA(cudaMalloc(&dtab, sizeof(double) * tab.size()), "dg_eval_points alloc");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(dtab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = (cudaError_t)dg::launch_eval_points(m, c, dtab, npts, out, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(dtab);
  if (e != cudaSuccess) return cuda_fail(e, "dg_eval_points");
  return DG_OK;
}

extern "C" dg_status dg_det_j(const dg_mesh *m, double *detj, void *stream) {
  if (!m || !detj) return fail(DG_EINVAL, "dg_det_j: null argument");
  if (dg_status dst = check_device(m, "dg_det_j")) return dst;
  DG_CUDA((cudaError_t)dg::launch_det_j(m, detj, stream), "dg_det_j");
  return DG_OK;
}

// the reference points (r[k], s[k]) checked and packed for the device
static dg_status ref_points(const char *who, int npts, const double *r, const double *s, std::vector<double> &rs) {
  if (npts < 1 || npts > 1 << 20) return fail(DG_EINVAL, "%s: npts=%d", who, npts);
  rs.resize(2 * (size_t)npts);
  for (int k = 0; k < npts; ++k) {
    if (!(r[k] >= 0.0 && s[k] >= 0.0 && r[k] + s[k] < 1.0))
      return fail(DG_EINVAL, "%s: point %d = (%g, %g) is not inside the reference triangle", who, k, r[k], s[k]);
    rs[2 * k] = r[k];
    rs[2 * k + 1] = s[k];
  }
  return DG_OK;
}

extern "C" dg_status dg_map_points(const dg_mesh *m, int npts, const double *r, const double *s, double *xy,
                                   void *stream) {
  if (!m || !r || !s || !xy) return fail(DG_EINVAL, "dg_map_points: null argument");
  if (dg_status dst = check_device(m, "dg_map_points")) return dst;
  std::vector<double> rs;
  if (dg_status st = ref_points("dg_map_points", npts, r, s, rs)) return st;
  double *drs = nullptr;
  DG_CUDA(cudaMalloc(&drs, sizeof(double) * rs.size()), "dg_map_points alloc");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(drs, rs.data(), sizeof(double) * rs.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = (cudaError_t)dg::launch_map_points(m, drs, npts, xy, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(drs);
  if (e != cudaSuccess) return cuda_fail(e, "dg_map_points");
  return DG_OK;
}

extern "C" dg_status dg_l2_error(const dg_mesh *m, int npts, const double *r, const double *s, const double *w,
                                 const double *c, const double *exact, int var, double *err_out, void *stream) {
  if (!m || !r || !s || !w || !c || !exact || !err_out) return fail(DG_EINVAL, "dg_l2_error: null argument");
  if (dg_status dst = check_device(m, "dg_l2_error")) return dst;
  if (var < 0 || var >= dg::M) return fail(DG_EINVAL, "dg_l2_error: var=%d", var);
  std::vector<double> rs;
  if (dg_status st = ref_points("dg_l2_error", npts, r, s, rs)) return st;
  // basis values at the points, the weights, block partials and the result in one buffer
  const int nb = 256;
  std::vector<double> host((size_t)npts * m->np + npts);
  for (int k = 0; k < npts; ++k) {
    dubiner(m->p, (real)r[k], (real)s[k], &host[(size_t)k * m->np], nullptr, nullptr);
    host[(size_t)npts * m->np + k] = w[k];
  }
  double *buf = nullptr;
  DG_CUDA(cudaMalloc(&buf, sizeof(double) * (host.size() + nb + 1)), "dg_l2_error alloc");
  cudaStream_t st = (cudaStream_t)stream;
  double *tab = buf, *dw = buf + (size_t)npts * m->np, *partial = dw + npts, *res = partial + nb;
  cudaError_t e = cudaMemcpyAsync(buf, host.data(), sizeof(double) * host.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = (cudaError_t)dg::launch_l2_error(m, c, exact, tab, dw, npts, var, partial, nb, res, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(err_out, res, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_fail(e, "dg_l2_error");
  return DG_OK;
}

extern "C" dg_status dg_project_ic(dg_mesh *m, const double *u, double *c, void *stream) {
  if (!m || !u || !c) return fail(DG_EINVAL, "dg_project_ic: null argument");
  if (dg_status dst = check_device(m, "dg_project_ic")) return dst;
  DG_CUDA((cudaError_t)timed(m, DG_K_PROJECT, stream, [&] { return dg::launch_project(m, u, c, stream); }),
          "dg_project_ic");
  return DG_OK;
}

static dg_status check_prec(dg_precision prec, const char *who) {
  if (prec == DG_FP64 || prec == DG_TF32X1 || prec == DG_TF32X3) return DG_OK;
  return fail(DG_EINVAL, "%s: unknown precision %d", who, (int)prec);
}

// element kernel of the chosen precision
// The three launches of a stage in either precision: the first traces (when
// asked for), the edge fluxes, and the element kernel.  The mixed modes keep
// their float32 traces and fluxes in the float64 buffers' storage.
static int launch_traces_p(dg_mesh *m, dg_precision prec, const double *c, void *stream) {
  if (prec == DG_FP64) return dg::launch_traces(m, c, m->trace, stream);
  const dg::MixedBuffers b = dg::mixed_buffers(m, m->trace, m->fhat);
  return dg::launch_element_tc(m, prec == DG_TF32X3 ? 1 : 0, c, nullptr, nullptr, b.trace, nullptr, nullptr, 0.0,
                               0.0, 0.0, 2, stream);
}
static int launch_face_p(dg_mesh *m, dg_precision prec, void *stream) {
  if (prec == DG_FP64) return dg::launch_face_flux(m, m->trace, m->fhat, stream);
  return dg::launch_face_flux_mixed(m, dg::mixed_buffers(m, m->trace, m->fhat), stream);
}
static int launch_elem(dg_mesh *m, dg_precision prec, const double *c, const double *u0, double *out,
                       bool traces, const dg::StageUpdate &su, int mode, void *stream) {
  if (prec == DG_FP64)
    return dg::launch_element(m, c, u0, out, traces ? m->trace : nullptr, m->fhat, su, mode, stream);
  const dg::MixedBuffers b = dg::mixed_buffers(m, m->trace, m->fhat);
  return dg::launch_element_tc(m, prec == DG_TF32X3 ? 1 : 0, c, u0, out, traces ? b.trace : nullptr, b.fhat,
                               b.fmean, su, mode, stream);
}

extern "C" dg_status dg_rhs(dg_mesh *m, const double *c, double *r, dg_precision prec, void *stream) {
  if (!m || !c || !r) return fail(DG_EINVAL, "dg_rhs: null argument");
  if (dg_status dst = check_device(m, "dg_rhs")) return dst;
  if (c == r) return fail(DG_EINVAL, "dg_rhs: c and r alias");
  dg_status st = check_prec(prec, "dg_rhs");
  if (st != DG_OK) return st;
  if (!m->bstate_set) return fail(DG_EINVAL, "dg_rhs: the mesh has DG_BC_STATE faces and no boundary state was set");
  DG_CUDA((cudaError_t)timed(m, DG_K_TRACES, stream, [&] { return launch_traces_p(m, prec, c, stream); }),
          "dg_rhs traces");
  DG_CUDA((cudaError_t)timed(m, DG_K_FACE, stream, [&] { return launch_face_p(m, prec, stream); }),
          "dg_rhs edge flux");
  DG_CUDA((cudaError_t)timed(m, DG_K_ELEMENT, stream, [&] {
            return launch_elem(m, prec, c, nullptr, r, false, dg::shu_osher(0.0, 0.0, 0.0), 0, stream);
          }), "dg_rhs element");
  return DG_OK;
}

static dg_status check_method(dg_rk_method method, const char *who) {
  if (method == DG_SSP_RK3 || method == DG_RK2 || method == DG_RK4) return DG_OK;
  return fail(DG_EINVAL, "%s: unknown Runge-Kutta method %d", who, (int)method);
}

// One step of the chosen Runge-Kutta method; on entry m->trace holds the traces
// of c when traces_valid.  Every stage is an edge-flux launch and an element
// launch; each element launch also writes the traces of its output, which the
// next stage (or step) reads.
static dg_status rk_step_one(dg_mesh *m, double *c, double dt, bool traces_valid, dg_rk_method method,
                             dg_precision prec, void *stream) {
  using namespace dg;
  auto face = [&](const char *what) -> dg_status {
    DG_CUDA((cudaError_t)timed(m, DG_K_FACE, stream, [&] { return launch_face_p(m, prec, stream); }), what);
    return DG_OK;
  };
  auto elem = [&](const double *cin, const double *u0, double *out, const StageUpdate &su,
                  const char *what) -> dg_status {
    DG_CUDA((cudaError_t)timed(m, DG_K_ELEMENT, stream, [&] {
              return launch_elem(m, prec, cin, u0, out, true, su, 1, stream);
            }), what);
    return DG_OK;
  };
  // With the limiter on (Section 4.3.5, p = 1) every stage value and the new
  // state are limited; the limiter reads the traces the element kernel wrote and
  // rewrites those of the elements it limits, for the next stage.
  auto stage = [&](const double *cin, const double *u0, double *out, const StageUpdate &su,
                   const char *what) -> dg_status {
    dg_status st = face(what);
    if (st != DG_OK) return st;
    if ((st = elem(cin, u0, out, su, what)) != DG_OK || !m->limiter) return st;
    DG_CUDA((cudaError_t)timed(m, DG_K_OTHER, stream, [&] { return launch_limit(m, out, m->trace, 1, stream); }),
            what);
    return DG_OK;
  };
  dg_status st;
  // mixed modes: the first stage's traces on the tensor cores, like the traces
  // the element kernel writes for the later stages
  if (!traces_valid)
    DG_CUDA((cudaError_t)timed(m, DG_K_TRACES, stream, [&] { return launch_traces_p(m, prec, c, stream); }),
            "rk traces");
  if (method != DG_SSP_RK3 && method != DG_RK2 && method != DG_RK4) return fail(DG_EINVAL, "rk step: unknown method");
  const int ns = rk_num_stages(method);
  for (int i = 0; i < ns; ++i) {
    const RkStage rs = rk_stage(method, i, dt, c, m->stage, m->rk_acc);
    if ((st = stage(rs.cin, rs.u0, rs.out, rs.su, "rk stage")) != DG_OK) return st;
  }
  return DG_OK;
}

// Steps per captured graph.  Replaying a graph runs its launches back to back,
// which is what small meshes (a few microseconds of work per kernel) need.
constexpr int kGraphSteps = 16;

// The cached graph of kGraphSteps steps for (c, dt, prec), capturing it if the
// key changed; nullptr if capture is unavailable (plain launches are used).
static cudaGraphExec_t step_graph(dg_mesh *m, double *c, double dt, dg_rk_method method, dg_precision prec) {
  if (!m->graph) m->graph = new (std::nothrow) dg::GraphCache();
  dg::GraphCache *g = m->graph;
  if (!g || g->broken) return nullptr;
  if (g->exec && g->c == c && g->dt == dt && g->prec == (int)prec && g->method == (int)method &&
      g->steps == kGraphSteps)
    return g->exec;
  if (g->exec) { cudaGraphExecDestroy(g->exec); g->exec = nullptr; }
  if (!g->stream && cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess) g->stream = nullptr;
  if (g->stream && !g->ready && cudaEventCreateWithFlags(&g->ready, cudaEventDisableTiming) != cudaSuccess) g->ready = nullptr;
  if (g->stream && !g->done && cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming) != cudaSuccess) g->done = nullptr;
  if (!g->stream || !g->ready || !g->done) { cudaGetLastError(); g->broken = true; return nullptr; }
  cudaGraph_t graph = nullptr;
  bool ok = cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeRelaxed) == cudaSuccess;
  if (ok) {
    for (int i = 0; i < kGraphSteps && ok; ++i) ok = rk_step_one(m, c, dt, true, method, prec, g->stream) == DG_OK;
    ok = (cudaStreamEndCapture(g->stream, &graph) == cudaSuccess) && ok && graph;
  }
  if (ok) ok = cudaGraphInstantiate(&g->exec, graph, 0) == cudaSuccess;
  if (graph) cudaGraphDestroy(graph);
  if (!ok) {
    cudaGetLastError();
    g->exec = nullptr;
    g->broken = true;
    g_err.clear();
    return nullptr;
  }
  g->c = c; g->dt = dt; g->prec = (int)prec; g->method = (int)method; g->steps = kGraphSteps;
  return g->exec;
}

// whether the mesh's device runs cooperative launches (every block of the grid
// resident at once), asked once per device
static bool coop_capable(const dg_mesh *m) {
  static dg::PerDevice asked, yes;
  if (!asked.test(m->device)) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrCooperativeLaunch, m->device) != cudaSuccess) {
      cudaGetLastError();
      v = 0;
    }
    if (v) yes.set(m->device);
    asked.set(m->device);
  }
  return yes.test(m->device);
}

extern "C" dg_status dg_rk_step_method(dg_mesh *m, double *c, double dt, int nsteps, dg_rk_method method,
                                       dg_precision prec, void *stream) {
  if (!m || !c) return fail(DG_EINVAL, "dg_rk_step: null argument");
  if (dg_status dst = check_device(m, "dg_rk_step")) return dst;
  if (nsteps < 0) return fail(DG_EINVAL, "dg_rk_step: nsteps < 0");
  if (!std::isfinite(dt)) return fail(DG_EINVAL, "dg_rk_step: dt is not finite");
  dg_status st = check_prec(prec, "dg_rk_step");
  if (st != DG_OK) return st;
  if ((st = check_method(method, "dg_rk_step")) != DG_OK) return st;
  if (!m->bstate_set)
    return fail(DG_EINVAL, "dg_rk_step: the mesh has DG_BC_STATE faces and no boundary state was set");
  if (m->limiter && prec != DG_FP64)
    return fail(DG_ENOTIMPL, "dg_rk_step: the limiter runs with the float64 path only");
  if (method == DG_RK4 && !m->rk_acc && nsteps > 0) {
    cudaError_t e = cudaMalloc(&m->rk_acc, sizeof(double) * m->N * dg::M * m->np);
    if (e != cudaSuccess) { cudaGetLastError(); m->rk_acc = nullptr; return fail(DG_ENOMEM, "dg_rk_step: RK4 buffer"); }
  }
  // a small mesh in float64: the whole call in one launch of the fused stepper
  // (after the traces of c), the limiter included when it is on
  if (nsteps > 0 && prec == DG_FP64 && m->small_stepper && dg::small_rk_fits(m) && coop_capable(m)) {
    DG_CUDA((cudaError_t)timed(m, DG_K_TRACES, stream, [&] { return dg::launch_traces(m, c, m->trace, stream); }),
            "dg_rk_step traces");
    DG_CUDA((cudaError_t)timed(m, DG_K_STEPPER, stream,
                               [&] { return dg::launch_rk_small(m, c, dt, nsteps, (int)method, stream); }),
            "dg_rk_step fused small-mesh stepper");
    return DG_OK;
  }
  int done = 0;
  if (nsteps > 0) {
    if ((st = rk_step_one(m, c, dt, false, method, prec, stream)) != DG_OK) return st;
    done = 1;
  }
  // whole chunks of steps as a replayed CUDA graph (not while per-kernel timing is on)
  if (nsteps - done >= kGraphSteps && !(m->timing && m->timing->on)) {
    cudaGraphExec_t exec = step_graph(m, c, dt, method, prec);
    if (exec) {
      dg::GraphCache *g = m->graph;
      cudaStream_t s = (cudaStream_t)stream;
      DG_CUDA(cudaEventRecord(g->ready, s), "dg_rk_step graph order");
      DG_CUDA(cudaStreamWaitEvent(g->stream, g->ready, 0), "dg_rk_step graph order");
      while (nsteps - done >= kGraphSteps) {
        DG_CUDA(cudaGraphLaunch(exec, g->stream), "dg_rk_step graph launch");
        done += kGraphSteps;
      }
      DG_CUDA(cudaEventRecord(g->done, g->stream), "dg_rk_step graph order");
      DG_CUDA(cudaStreamWaitEvent(s, g->done, 0), "dg_rk_step graph order");
    }
  }
  for (; done < nsteps; ++done)
    if ((st = rk_step_one(m, c, dt, true, method, prec, stream)) != DG_OK) return st;
  return DG_OK;
}

extern "C" dg_status dg_set_small_mesh_stepper(dg_mesh *m, int enable) {
  if (!m) return fail(DG_EINVAL, "dg_set_small_mesh_stepper: null mesh");
  m->small_stepper = enable != 0;
  return DG_OK;
}

extern "C" dg_status dg_set_limiter(dg_mesh *m, int enable) {
  if (!m) return fail(DG_EINVAL, "dg_set_limiter: null mesh");
  if (enable && m->p != 1) return fail(DG_EINVAL, "dg_set_limiter: the Barth-Jespersen limiter is for p = 1 (p = %d)", m->p);
  if ((enable != 0) != (m->limiter != 0) && m->graph && m->graph->exec) {
    cudaGraphExecDestroy(m->graph->exec);    // captured with the other setting
    m->graph->exec = nullptr;
  }
  m->limiter = enable != 0;
  return DG_OK;
}

extern "C" dg_status dg_limit(dg_mesh *m, double *c, void *stream) {
  if (!m || !c) return fail(DG_EINVAL, "dg_limit: null argument");
  if (dg_status dst = check_device(m, "dg_limit")) return dst;
  if (m->p != 1) return fail(DG_EINVAL, "dg_limit: the Barth-Jespersen limiter is for p = 1 (p = %d)", m->p);
  DG_CUDA((cudaError_t)timed(m, DG_K_OTHER, stream, [&] { return dg::launch_limit(m, c, nullptr, 0, stream); }),
          "dg_limit");
  return DG_OK;
}

extern "C" dg_status dg_rk_step(dg_mesh *m, double *c, double dt, int nsteps, dg_precision prec,
                                void *stream) {
  return dg_rk_step_method(m, c, dt, nsteps, DG_SSP_RK3, prec, stream);
}

// One float64 SSP-RK3 step on the device state c whose new state is also copied
// into c_host: the last stage's element launch is split into chunks of whole
// waves of the element kernel, and each chunk's rows travel to the host on
// m->copy_stream while the next chunk computes (the same launches otherwise,
// and the same bits: an element's arithmetic does not depend on its tile).
static dg_status ssp_step_copy_out(dg_mesh *m, double *c, double dt, double *c_host, void *stream) {
  using namespace dg;
  cudaStream_t s = (cudaStream_t)stream;
  if (!m->copy_stream) {
    if (cudaStreamCreateWithFlags(&m->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->copy_ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->copy_ev[1], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return fail(DG_ECUDA, "dg_rk_step_host: copy stream");
    }
  }
  auto face = [&]() -> dg_status {
    DG_CUDA((cudaError_t)timed(m, DG_K_FACE, stream, [&] { return launch_face_flux(m, m->trace, m->fhat, stream); }),
            "dg_rk_step_host flux");
    return DG_OK;
  };
  dg_status st;
  for (int i = 0; i < 2; ++i) {
    const RkStage rs = rk_stage(DG_SSP_RK3, i, dt, c, m->stage, m->rk_acc);
    if ((st = face()) != DG_OK) return st;
    DG_CUDA((cudaError_t)timed(m, DG_K_ELEMENT, stream, [&] {
              return launch_element(m, rs.cin, rs.u0, rs.out, m->trace, m->fhat, rs.su, 1, stream);
            }), "dg_rk_step_host stage");
  }
  if ((st = face()) != DG_OK) return st;
  const RkStage rs = rk_stage(DG_SSP_RK3, 2, dt, c, m->stage, m->rk_acc);
  int wave_tiles = 0, eb = 0;
  DG_CUDA((cudaError_t)element_wave(m, &wave_tiles, &eb), "dg_rk_step_host wave");
  const int64_t wave = (int64_t)wave_tiles * eb;
  const int64_t waves = (m->N + wave - 1) / wave;
  const int64_t chunk = std::max<int64_t>(1, waves / 4) * wave;
  const size_t row = (size_t)M * m->np;
  for (int64_t e0 = 0; e0 < m->N; e0 += chunk) {
    const int64_t e1 = std::min<int64_t>(m->N, e0 + chunk);
    DG_CUDA((cudaError_t)timed(m, DG_K_ELEMENT, stream, [&] {
              return launch_element(m, rs.cin, rs.u0, rs.out, m->trace, m->fhat, rs.su, 1, stream, e0, e1);
            }), "dg_rk_step_host last stage");
    DG_CUDA(cudaEventRecord(m->copy_ev[0], s), "dg_rk_step_host order");
    DG_CUDA(cudaStreamWaitEvent(m->copy_stream, m->copy_ev[0], 0), "dg_rk_step_host order");
    DG_CUDA(cudaMemcpyAsync(c_host + e0 * row, c + e0 * row, sizeof(double) * (e1 - e0) * row,
                            cudaMemcpyDeviceToHost, m->copy_stream), "dg_rk_step_host D2H");
  }
  DG_CUDA(cudaEventRecord(m->copy_ev[1], m->copy_stream), "dg_rk_step_host order");
  DG_CUDA(cudaStreamWaitEvent(s, m->copy_ev[1], 0), "dg_rk_step_host order");
  return DG_OK;
}

extern "C" dg_status dg_rk_step_host(dg_mesh *m, double *c_host, double dt, int nsteps,
                                     dg_precision prec, void *stream) {
  if (!m || !c_host) return fail(DG_EINVAL, "dg_rk_step_host: null argument");
  if (dg_status dst = check_device(m, "dg_rk_step_host")) return dst;
  size_t bytes = sizeof(double) * m->N * dg::M * m->np;
  if (!m->host_state) {
    cudaError_t e = cudaMalloc(&m->host_state, bytes);
    if (e != cudaSuccess) { cudaGetLastError(); m->host_state = nullptr; return fail(DG_ENOMEM, "dg_rk_step_host: cudaMalloc"); }
  }
  cudaStream_t s = (cudaStream_t)stream;
  // c_host in page-locked memory the device reaches (NVLink-C2C on this part):
  // the first kernel (the traces of c) reads it in place and writes the device
  // copy the steps run on, so the copy in travels while the traces are formed.
  // The copy out of the new state runs in chunks behind the last stage
  // (ssp_step_copy_out).  The same arithmetic as below, so the same results.
  // (Float64 without the limiter, on meshes the fused small-mesh stepper does
  // not take.  Writing the new state from the last stage straight into host
  // memory measured slower than copies.)
  if (nsteps >= 1 && prec == DG_FP64 && !m->limiter && m->bstate_set &&
      !(m->small_stepper && dg::small_rk_fits(m))) {
    cudaPointerAttributes pa;
    double *dev = nullptr;
    if (cudaPointerGetAttributes(&pa, c_host) == cudaSuccess) {
      if (pa.type == cudaMemoryTypeHost && pa.devicePointer) dev = static_cast<double *>(pa.devicePointer);
    } else {
      cudaGetLastError();
    }
    if (dev && std::isfinite(dt)) {
      DG_CUDA((cudaError_t)timed(m, DG_K_TRACES, stream, [&] {
                return dg::launch_traces(m, dev, m->trace, stream, m->host_state);
              }), "dg_rk_step_host traces");
      for (int i = 0; i + 1 < nsteps; ++i) {
        dg_status st = rk_step_one(m, m->host_state, dt, true, DG_SSP_RK3, prec, stream);
        if (st != DG_OK) return st;
      }
      dg_status st = ssp_step_copy_out(m, m->host_state, dt, c_host, stream);
      if (st != DG_OK) return st;
      DG_CUDA(cudaStreamSynchronize(s), "dg_rk_step_host sync");
      return DG_OK;
    }
  }
  DG_CUDA(cudaMemcpyAsync(m->host_state, c_host, bytes, cudaMemcpyHostToDevice, s), "dg_rk_step_host H2D");
  dg_status st = dg_rk_step(m, m->host_state, dt, nsteps, prec, stream);
  if (st != DG_OK) return st;
  DG_CUDA(cudaMemcpyAsync(c_host, m->host_state, bytes, cudaMemcpyDeviceToHost, s), "dg_rk_step_host D2H");
  DG_CUDA(cudaStreamSynchronize(s), "dg_rk_step_host sync");
  return DG_OK;
}

extern "C" dg_status dg_conserved_totals(dg_mesh *m, const double *c, double out[4], void *stream) {
  if (!m || !c || !out) return fail(DG_EINVAL, "dg_conserved_totals: null argument");
  if (dg_status dst = check_device(m, "dg_conserved_totals")) return dst;
  cudaStream_t s = (cudaStream_t)stream;
  DG_CUDA((cudaError_t)timed(m, DG_K_TOTALS, stream, [&] { return dg::launch_totals(m, c, m->totals_dev, stream); }),
          "dg_conserved_totals");
  DG_CUDA(cudaMemcpyAsync(out, m->totals_dev, sizeof(double) * dg::M, cudaMemcpyDeviceToHost, s),
          "dg_conserved_totals D2H");
  DG_CUDA(cudaStreamSynchronize(s), "dg_conserved_totals sync");
  return DG_OK;
}

// adjoint work space: 5 states and 2 trace blocks, allocated on first use
static dg_status adjoint_buffers(dg_mesh *m, const char *who) {
  const size_t S = (size_t)m->N * dg::M * m->np;
  const size_t TR = (size_t)m->N * 3 * m->ne * dg::M;
  const size_t need = 5 * S + 2 * TR;
  if (m->adj_doubles < need) {
    cudaFree(m->adj_buf);
    m->adj_buf = nullptr;
    m->adj_doubles = 0;
    cudaError_t e = cudaMalloc(&m->adj_buf, sizeof(double) * need);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(DG_ENOMEM, "%s: cudaMalloc", who); }
    m->adj_doubles = need;
  }
  return DG_OK;
}

extern "C" dg_status dg_rhs_adjoint(dg_mesh *m, const double *c, const double *lam, double *out, void *stream) {
  using namespace dg;
  if (!m || !c || !lam || !out) return fail(DG_EINVAL, "dg_rhs_adjoint: null argument");
  if (dg_status dst = check_device(m, "dg_rhs_adjoint")) return dst;
  if (out == c || out == lam) return fail(DG_EINVAL, "dg_rhs_adjoint: out aliases an input");
  dg_status st = adjoint_buffers(m, "dg_rhs_adjoint");
  if (st != DG_OK) return st;
  const size_t S = (size_t)m->N * M * m->np, TR = (size_t)m->N * 3 * m->ne * M;
  double *uvol = m->adj_buf + 4 * S, *G = m->adj_buf + 5 * S, *TB = G + TR;
  DG_CUDA((cudaError_t)timed(m, DG_K_ADJOINT, stream, [&] {
            return launch_rhs_vjp(m, c, lam, uvol, G, m->trace, TB, nullptr, nullptr, nullptr, 0.0, 0.0, 0.0, 1.0,
                                  out, stream);
          }), "dg_rhs_adjoint");
  return DG_OK;
}

// The reverse sweep of one SSP-RK3 step from c_n, given its stage values u1, u2:
// c_{n+1} = 1/3 c_n + 2/3 (u2 + dt R(u2)), u2 = 3/4 c_n + 1/4 (u1 + dt R(u1)),
// u1 = c_n + dt R(c_n), transposed stage by stage.
static dg_status adjoint_sweep(dg_mesh *m, const double *c_n, const double *u1, const double *u2, double dt,
                               const double *lam_np1, double *lam_n, void *stream) {
  using namespace dg;
  const size_t S = (size_t)m->N * M * m->np;           // one state
  const size_t TR = (size_t)m->N * 3 * m->ne * M;       // one trace block
  double *b1 = m->adj_buf + 2 * S, *b2 = b1 + S, *uvol = b2 + S;
  double *G = uvol + S, *TB = G + TR;
  auto vjp = [&](const double *u, const double *lam, const double *X, const double *Y, const double *Z,
                 double x0, double x1, double x2, double s, double *out, const char *what) -> dg_status {
    DG_CUDA((cudaError_t)timed(m, DG_K_ADJOINT, stream, [&] {
              return launch_rhs_vjp(m, u, lam, uvol, G, m->trace, TB, X, Y, Z, x0, x1, x2, s, out, stream);
            }), what);
    return DG_OK;
  };
  dg_status st;
  // b2 = 2/3 (lam + dt R'(u2)^T lam)
  if ((st = vjp(u2, lam_np1, lam_np1, nullptr, nullptr, 2.0 / 3.0, 0, 0, 2.0 / 3.0 * dt, b2, "adjoint u2")) != DG_OK)
    return st;
  // b1 = 1/4 (b2 + dt R'(u1)^T b2)
  if ((st = vjp(u1, b2, b2, nullptr, nullptr, 0.25, 0, 0, 0.25 * dt, b1, "adjoint u1")) != DG_OK) return st;
  // lam_n = 1/3 lam + 3/4 b2 + b1 + dt R'(c_n)^T b1
  if ((st = vjp(c_n, b1, lam_np1, b2, b1, 1.0 / 3.0, 0.75, 1.0, dt, lam_n, "adjoint c_n")) != DG_OK) return st;
  return DG_OK;
}

// The forward stages of one SSP-RK3 step from c: u1 = c + dt R(c) and
// u2 = 3/4 c + 1/4 (u1 + dt R(u1)); with cnew, also cnew = 1/3 c + 2/3 (u2 + dt R(u2))
// (cnew may be c).  The same launches, in the same order, as a float64 dg_rk_step
// step, so the values are the same bits.
static dg_status forward_stages(dg_mesh *m, const double *c, double dt, double *u1, double *u2, double *cnew,
                                void *stream) {
  using namespace dg;
  DG_CUDA((cudaError_t)timed(m, DG_K_TRACES, stream, [&] { return launch_traces(m, c, m->trace, stream); }),
          "stages traces");
  DG_CUDA((cudaError_t)timed(m, DG_K_FACE, stream, [&] { return launch_face_flux(m, m->trace, m->fhat, stream); }),
          "stage 1 flux");
  DG_CUDA((cudaError_t)timed(m, DG_K_ELEMENT, stream, [&] {
            return launch_element(m, c, nullptr, u1, m->trace, m->fhat, dt, 0.0, 1.0, 1, stream);
          }), "stage 1");
  DG_CUDA((cudaError_t)timed(m, DG_K_FACE, stream, [&] { return launch_face_flux(m, m->trace, m->fhat, stream); }),
          "stage 2 flux");
  DG_CUDA((cudaError_t)timed(m, DG_K_ELEMENT, stream, [&] {
            return launch_element(m, u1, c, u2, cnew ? m->trace : nullptr, m->fhat, dt, 0.75, 0.25, 1, stream);
          }), "stage 2");
  if (!cnew) return DG_OK;
  DG_CUDA((cudaError_t)timed(m, DG_K_FACE, stream, [&] { return launch_face_flux(m, m->trace, m->fhat, stream); }),
          "stage 3 flux");
  DG_CUDA((cudaError_t)timed(m, DG_K_ELEMENT, stream, [&] {
            return launch_element(m, u2, c, cnew, m->trace, m->fhat, dt, 1.0 / 3.0, 2.0 / 3.0, 1, stream);
          }), "stage 3");
  return DG_OK;
}

static dg_status adjoint_checks(dg_mesh *m, const void *c_n, double dt, const void *lam_np1, const void *lam_n,
                                const char *who) {
  if (!m || !c_n || !lam_np1 || !lam_n) return fail(DG_EINVAL, "%s: null argument", who);
  if (dg_status dst = check_device(m, who)) return dst;
  if (lam_n == lam_np1 || lam_n == c_n) return fail(DG_EINVAL, "%s: lam_n aliases an input", who);
  if (!std::isfinite(dt)) return fail(DG_EINVAL, "%s: dt is not finite", who);
  if (m->limiter) return fail(DG_ENOTIMPL, "%s: the limited step has no adjoint here (the limiter is off by default)", who);
  return adjoint_buffers(m, who);
}

extern "C" dg_status dg_adjoint_step(dg_mesh *m, const double *c_n, double dt, const double *lam_np1,
                                     double *lam_n, void *stream) {
  dg_status st = adjoint_checks(m, c_n, dt, lam_np1, lam_n, "dg_adjoint_step");
  if (st != DG_OK) return st;
  const size_t S = (size_t)m->N * dg::M * m->np;
  double *u1 = m->adj_buf, *u2 = u1 + S;
  // the forward stages from c_n, then the reverse sweep
  if ((st = forward_stages(m, c_n, dt, u1, u2, nullptr, stream)) != DG_OK) return st;
  return adjoint_sweep(m, c_n, u1, u2, dt, lam_np1, lam_n, stream);
}

extern "C" dg_status dg_rk_step_stages(dg_mesh *m, double *c, double dt, double *u1, double *u2, void *stream) {
  if (!m || !c || !u1 || !u2) return fail(DG_EINVAL, "dg_rk_step_stages: null argument");
  if (dg_status dst = check_device(m, "dg_rk_step_stages")) return dst;
  if (u1 == u2 || u1 == c || u2 == c) return fail(DG_EINVAL, "dg_rk_step_stages: c, u1 and u2 must be distinct");
  if (!std::isfinite(dt)) return fail(DG_EINVAL, "dg_rk_step_stages: dt is not finite");
  if (!m->bstate_set)
    return fail(DG_EINVAL, "dg_rk_step_stages: the mesh has DG_BC_STATE faces and no boundary state was set");
  if (m->limiter) return fail(DG_ENOTIMPL, "dg_rk_step_stages: not with the limiter on");
  return forward_stages(m, c, dt, u1, u2, c, stream);
}

extern "C" dg_status dg_adjoint_step_stages(dg_mesh *m, const double *c_n, const double *u1, const double *u2,
                                            double dt, const double *lam_np1, double *lam_n, void *stream) {
  dg_status st = adjoint_checks(m, c_n, dt, lam_np1, lam_n, "dg_adjoint_step_stages");
  if (st != DG_OK) return st;
  if (!u1 || !u2) return fail(DG_EINVAL, "dg_adjoint_step_stages: null argument");
  if (lam_n == u1 || lam_n == u2) return fail(DG_EINVAL, "dg_adjoint_step_stages: lam_n aliases an input");
  return adjoint_sweep(m, c_n, u1, u2, dt, lam_np1, lam_n, stream);
}

extern "C" dg_status dg_set_timing(dg_mesh *m, int enable) {
  if (!m || !m->timing) return fail(DG_EINVAL, "dg_set_timing: null mesh");
  dg::Timing *t = m->timing;
  if (t->used) cudaDeviceSynchronize();
  t->on = enable != 0;
  t->used = 0;
  for (int k = 0; k < DG_NKINDS; ++k) { t->ms[k] = 0.0; t->launches[k] = 0; }
  return DG_OK;
}

extern "C" dg_status dg_kernel_times(dg_mesh *m, double ms[8], int64_t launches[8]) {
  if (!m || !m->timing || !ms || !launches) return fail(DG_EINVAL, "dg_kernel_times: null argument");
  dg::Timing *t = m->timing;
  for (size_t i = 0; i < t->used; ++i) {
    dg::Timing::Rec &r = t->pool[i];
    DG_CUDA(cudaEventSynchronize(r.b), "dg_kernel_times sync");
    float e = 0.f;
    DG_CUDA(cudaEventElapsedTime(&e, r.a, r.b), "dg_kernel_times elapsed");
    t->ms[r.kind] += (double)e;
    t->launches[r.kind] += 1;
  }
  t->used = 0;
  for (int k = 0; k < DG_NKINDS; ++k) { ms[k] = t->ms[k]; launches[k] = t->launches[k]; }
  return DG_OK;
}

extern "C" dg_status dg_probe_fma_rate(double *fp64_tflops, double *fp32_tflops, void *stream) {
  int dev = 0, sms = 0;
  DG_CUDA(cudaGetDevice(&dev), "probe");
  DG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "probe");
  const int threads = 256, blocks = sms * 8;
  double *buf = nullptr;
  DG_CUDA(cudaMalloc(&buf, sizeof(double) * blocks * threads), "probe alloc");
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  dg_status st = DG_OK;
  for (int fp64 = 1; fp64 >= 0 && st == DG_OK; --fp64) {
    double *dst = fp64 ? fp64_tflops : fp32_tflops;
    if (!dst) continue;
    const int iters = fp64 ? 4096 : 65536;
    cudaError_t e = (cudaError_t)dg::launch_fma_probe(fp64, blocks, threads, iters / 8, buf, stream);  // warm-up
    if (e == cudaSuccess) {
      cudaEventRecord(a, s);
      e = (cudaError_t)dg::launch_fma_probe(fp64, blocks, threads, iters, buf, stream);
      cudaEventRecord(b, s);
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e != cudaSuccess) { st = cuda_fail(e, "dg_probe_fma_rate"); break; }
    // 8 chains x iters FMAs x 2 flops per thread
    *dst = 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e-3) / 1e12;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(buf);
  return st;
}

extern "C" dg_status dg_device_status(dg_mesh *m, void *stream) {
  if (!m) return fail(DG_EINVAL, "dg_device_status: null mesh");
  cudaStream_t s = (cudaStream_t)stream;
  int flag = 0;
  DG_CUDA(cudaMemcpyAsync(&flag, m->err_flag, sizeof(int), cudaMemcpyDeviceToHost, s), "dg_device_status");
  DG_CUDA(cudaStreamSynchronize(s), "dg_device_status sync");
  if (flag) {
    DG_CUDA(cudaMemsetAsync(m->err_flag, 0, sizeof(int), s), "dg_device_status reset");
    DG_CUDA(cudaStreamSynchronize(s), "dg_device_status sync");
    if (flag & 4)
      return fail(DG_EMESH, "a kernel read a connectivity index out of range (checked in DG_DEBUG builds)");
    if (flag & 1)
      return fail(DG_ETIMEOUT, "a tensor-core wait in the mixed-precision kernel expired%s",
                  (flag & 2) ? "; a non-physical state was also met" : "");
    return fail(DG_ENONPHYS, "a non-physical state (rho <= 0 or p <= 0) was met at a quadrature point");
  }
  return DG_OK;
}

extern "C" dg_status dg_self_test(int64_t mismatches[4], void *stream) {
  if (!mismatches) return fail(DG_EINVAL, "dg_self_test: null argument");
  unsigned long long *bad = nullptr;
  DG_CUDA(cudaMalloc(&bad, 4 * sizeof(unsigned long long)), "dg_self_test alloc");
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long h[4] = {0, 0, 0, 0};
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof h, s);
  if (e == cudaSuccess) e = (cudaError_t)dg::launch_convert_check(1 << 20, bad, stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, bad, sizeof h, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(bad);
  if (e != cudaSuccess) return cuda_fail(e, "dg_self_test");
  for (int i = 0; i < 4; ++i) mismatches[i] = (int64_t)h[i];
  return DG_OK;
}

extern "C" dg_status dg_stable_dt(dg_mesh *m, const double *c, double cfl, double *dt_out, void *stream) {
  if (!m || !c || !dt_out) return fail(DG_EINVAL, "dg_stable_dt: null argument");
  if (dg_status dst = check_device(m, "dg_stable_dt")) return dst;
  if (!(cfl > 0.0)) return fail(DG_EINVAL, "dg_stable_dt: cfl must be positive");
  cudaStream_t s = (cudaStream_t)stream;
  double smax = 0.0;
  int flag = 0;
  DG_CUDA((cudaError_t)timed(m, DG_K_OTHER, stream, [&] { return dg::launch_wave_speed(m, c, m->totals_dev, stream); }),
          "dg_stable_dt");
  DG_CUDA(cudaMemcpyAsync(&smax, m->totals_dev, sizeof(double), cudaMemcpyDeviceToHost, s), "dg_stable_dt D2H");
  DG_CUDA(cudaMemcpyAsync(&flag, m->err_flag, sizeof(int), cudaMemcpyDeviceToHost, s), "dg_stable_dt D2H");
  DG_CUDA(cudaStreamSynchronize(s), "dg_stable_dt sync");
  if (flag & 2) {
    DG_CUDA(cudaMemset(m->err_flag, 0, sizeof(int)), "dg_stable_dt reset");
    return fail(DG_ENONPHYS, "dg_stable_dt: a non-physical state (rho <= 0 or p <= 0) was met");
  }
  if (!(smax > 0.0)) return fail(DG_ENONPHYS, "dg_stable_dt: no positive wave speed");
  *dt_out = cfl * m->rin_min / ((2 * m->p + 1) * smax);
  return DG_OK;
}
