// Host-side construction of the mesh tables and reference-cell tabulations.
//
// All tabulations are computed in FP64 and rounded once to FP32.  The routes are the
// library's own: Gauss-Legendre nodes and weights by the Golub-Welsch eigenproblem
// of the Legendre Jacobi matrix (cyclic Jacobi rotations), Legendre derivatives by
// the recurrence D^k P_{m+1} = D^k P_{m-1} + (2m+1) D^{k-1} P_m, the Taylor->Legendre
// corner maps by exact quadrature of the Taylor monomials, and the element semi-norm
// (eq. snorm) as a Gram matrix reduced by Cholesky factorisation.  The reference-cell
// tabulations are built in fixed-size stack arrays and written into a caller-provided
// DgTables (fill_dg_tables), with no allocation: the mesh path and the allocation-free
// step (noalloc.cu) share this one builder.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "cvweno_internal.cuh"

namespace cvw {
namespace {

constexpr int kMaxEig = kMaxGaussRule;  // largest eigenproblem: the largest Gauss rule

// Eigen-decomposition of a small symmetric matrix (n <= kMaxEig) by cyclic Jacobi
// rotations.  a is destroyed; eigenvalues to lam, eigenvectors as columns of v.
void jacobi_eigen(int n, double a[kMaxEig][kMaxEig], double lam[kMaxEig], double v[kMaxEig][kMaxEig]) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) v[i][j] = i == j ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) off += a[i][j] * a[i][j];
    if (off < 1e-300) break;
    for (int pi = 0; pi < n; ++pi) {
      for (int qi = pi + 1; qi < n; ++qi) {
        double apq = a[pi][qi];
        if (fabs(apq) < 1e-300) continue;
        double theta = (a[qi][qi] - a[pi][pi]) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          double akp = a[k][pi], akq = a[k][qi];
          a[k][pi] = c * akp - s * akq;
          a[k][qi] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          double apk = a[pi][k], aqk = a[qi][k];
          a[pi][k] = c * apk - s * aqk;
          a[qi][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = v[k][pi], vkq = v[k][qi];
          v[k][pi] = c * vkp - s * vkq;
          v[k][qi] = s * vkp + c * vkq;
        }
      }
    }
  }
  for (int i = 0; i < n; ++i) lam[i] = a[i][i];
}

// Golub-Welsch: nodes = eigenvalues of the symmetric Jacobi matrix of the Legendre
// recurrence, weights = 2 * (first eigenvector component)^2.  Ascending nodes; returns
// false (writing nothing) unless 1 <= n <= kMaxEig.
bool gauss_golub_welsch(int n, double* x, double* w) {
  if (n < 1 || n > kMaxEig) return false;
  double J[kMaxEig][kMaxEig] = {}, lam[kMaxEig], V[kMaxEig][kMaxEig];
  for (int k = 1; k < n; ++k) {
    double b = k / sqrt(4.0 * k * k - 1.0);
    J[k - 1][k] = J[k][k - 1] = b;
  }
  jacobi_eigen(n, J, lam, V);
  int idx[kMaxEig];
  for (int i = 0; i < n; ++i) idx[i] = i;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (lam[idx[j]] < lam[idx[i]]) { int t = idx[i]; idx[i] = idx[j]; idx[j] = t; }
  for (int i = 0; i < n; ++i) {
    x[i] = lam[idx[i]];
    double v0 = V[0][idx[i]];
    w[i] = 2.0 * v0 * v0;
  }
  // symmetrise (the rule is symmetric about 0)
  for (int i = 0; i < n / 2; ++i) {
    double xm = 0.5 * (x[n - 1 - i] - x[i]), wm = 0.5 * (w[i] + w[n - 1 - i]);
    x[i] = -xm;
    x[n - 1 - i] = xm;
    w[i] = w[n - 1 - i] = wm;
  }
  if (n % 2) x[n / 2] = 0.0;
  return true;
}

// D^k P_m(x) for m <= mmax, k <= kmax: out[k][m] (row stride mmax+1).
void legendre_derivs(double x, int mmax, int kmax, double* out) {
  int S = mmax + 1;
  for (int k = 0; k <= kmax; ++k)
    for (int m = 0; m <= mmax; ++m) out[k * S + m] = 0.0;
  out[0] = 1.0;
  if (mmax >= 1) out[1] = x;
  for (int m = 1; m < mmax; ++m) out[m + 1] = ((2.0 * m + 1.0) * x * out[m] - m * out[m - 1]) / (m + 1.0);
  for (int k = 1; k <= kmax; ++k) {
    if (mmax >= 1) out[k * S + 1] = (k == 1) ? 1.0 : 0.0;
    for (int m = 1; m < mmax; ++m)
      out[k * S + m + 1] = out[k * S + m - 1] + (2.0 * m + 1.0) * out[(k - 1) * S + m];
  }
}

double factorial(int k) {
  double f = 1.0;
  for (int i = 2; i <= k; ++i) f *= i;
  return f;
}

// The reference-cell tabulations of a dx x dy cell into *t (no allocation).
template <int DIM, int P>
cvweno_status fill_into(DgTables<DIM, P>* t, double dx, double dy) {
  using T = DgTables<DIM, P>;
  constexpr int N = T::N, ND = T::ND, NS = T::NS, NC = T::NC;
  memset(t, 0, sizeof(T));
  // h/dx and h/dy (h = sqrt(dx^2 + dy^2) in 2D, dx in 1D) from the aspect ratio alone:
  // every scaling below is a function of these two ratios, so square cells of any size
  // get bitwise the same tabulations (except tscale)
  const double ax = DIM == 2 ? sqrt(1.0 + (dy / dx) * (dy / dx)) : 1.0;
  const double ay = DIM == 2 ? sqrt((dx / dy) * (dx / dy) + 1.0) : 1.0;
  double gx[N], gw[N];
  gauss_golub_welsch(N, gx, gw);
  double tab[N * N];
  // E at +1
  legendre_derivs(1.0, P, P, tab);
  for (int k = 0; k < N; ++k)
    for (int mm = 0; mm < N; ++mm) t->E[k][mm] = (float)tab[k * N + mm];
  for (int q = 0; q < N; ++q) {
    legendre_derivs(gx[q], P, P, tab);
    for (int mm = 0; mm < N; ++mm) {
      t->B[q][mm] = (float)tab[mm];
      t->Bd[q][mm] = (float)tab[N + mm];
      for (int k = 0; k < N; ++k) t->Bk[k][q][mm] = (float)tab[k * N + mm];
    }
    t->w[q] = (float)gw[q];
  }
  // pointwise semi-norm weights and reference->physical scales
  for (int k = 0; k < ND; ++k) {
    int kx = k % N, ky = DIM == 2 ? k / N : 0;
    double sx = pow(2.0 * ax, 2 * kx), sy = DIM == 2 ? pow(2.0 * ay, 2 * ky) : 1.0;
    t->sigma[k] = (k == 0) ? 0.0f : (float)(sx * sy);
    t->tscale[k] = (float)(pow(2.0 / dx, kx) * (DIM == 2 ? pow(2.0 / dy, ky) : 1.0));
  }
  // 1D Gram blocks g_k[a][b] = int_{-1}^{1} D^k P_a D^k P_b, by an 8-point rule (exact)
  const int NG = 8;
  double qx[NG], qw[NG];
  gauss_golub_welsch(NG, qx, qw);
  double g[N * N * N] = {};  // [k][a][b]
  double tq[N * N];
  for (int q = 0; q < NG; ++q) {
    legendre_derivs(qx[q], P, P, tq);
    for (int k = 0; k < N; ++k)
      for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) g[(k * N + a) * N + b] += qw[q] * tq[k * N + a] * tq[k * N + b];
  }
  // element semi-norm Gram matrix on modes (eq. snorm), physical scaling folded in:
  // h^(2|k| - dim) (2/dx)^(2kx) (2/dy)^(2ky) |J| = (2h/dx)^(2kx) (2h/dy)^(2ky) |J| / h^dim
  // with |J| / h^dim = 1 / (4 ax ay) in 2D and 1 / (2 ax) in 1D
  double G[ND * ND] = {};
  for (int k = 1; k < ND; ++k) {
    int kx = k % N, ky = DIM == 2 ? k / N : 0;
    double rho = pow(2.0 * ax, 2 * kx) * (DIM == 2 ? pow(2.0 * ay, 2 * ky) : 1.0) /
                 (DIM == 2 ? 4.0 * ax * ay : 2.0 * ax);
    for (int a = 0; a < ND; ++a)
      for (int b = 0; b < ND; ++b) {
        int ax = a % N, ay = DIM == 2 ? a / N : 0, bx = b % N, by = DIM == 2 ? b / N : 0;
        double v = g[(kx * N + ax) * N + bx];
        if (DIM == 2) v *= g[(ky * N + ay) * N + by];
        G[a * ND + b] += rho * v;
      }
  }
  // Cholesky G[1:,1:] = R^T R, R upper triangular
  double R[NS * NS] = {};
  for (int j = 0; j < NS; ++j) {
    double s = G[(j + 1) * ND + (j + 1)];
    for (int k = 0; k < j; ++k) s -= R[k * NS + j] * R[k * NS + j];
    if (!(s > 0.0)) return CVWENO_ERR_ARG;
    R[j * NS + j] = sqrt(s);
    for (int i = j + 1; i < NS; ++i) {
      double v = G[(j + 1) * ND + (i + 1)];
      for (int k = 0; k < j; ++k) v -= R[k * NS + j] * R[k * NS + i];
      R[j * NS + i] = v / R[j * NS + j];
    }
  }
  for (int i = 0; i < NS; ++i)
    for (int j = 0; j < NS; ++j) t->R[i][j] = (float)R[i * NS + j];
  // Taylor->Legendre at corner s = -1, +1:  Gs[m][k] = (2m+1)/2 int P_m (xi - s)^k / k!
  double Gs[2][N][N];
  for (int si = 0; si < 2; ++si) {
    double s = si ? 1.0 : -1.0;
    for (int a = 0; a < N; ++a)
      for (int k = 0; k < N; ++k) {
        double acc = 0.0;
        for (int q = 0; q < NG; ++q) {
          legendre_derivs(qx[q], P, 0, tq);
          acc += qw[q] * tq[a] * pow(qx[q] - s, k) / factorial(k);
        }
        Gs[si][a][k] = 0.5 * (2 * a + 1) * acc;
      }
  }
  for (int l = 0; l < NC; ++l) {
    int sxi = l & 1, syi = (l >> 1) & 1;
    // C[a][k] for a, k in 1..ND-1, then A = R C
    double C[NS * NS];
    for (int a = 1; a < ND; ++a)
      for (int k = 1; k < ND; ++k) {
        int ax = a % N, ay = DIM == 2 ? a / N : 0, kx = k % N, ky = DIM == 2 ? k / N : 0;
        double v = Gs[sxi][ax][kx];
        if (DIM == 2) v *= Gs[syi][ay][ky];
        C[(a - 1) * NS + (k - 1)] = v;
      }
    for (int i = 0; i < NS; ++i)
      for (int j = 0; j < NS; ++j) {
        double acc = 0.0;
        for (int k = i; k < NS; ++k) acc += R[i * NS + k] * C[k * NS + j];
        t->A[l][i][j] = (float)acc;
      }
  }
  return CVWENO_OK;
}

// The mesh's own copy of its tabulations (owned by the mesh).
template <int DIM, int P>
cvweno_status fill(cvweno_mesh m) {
  using T = DgTables<DIM, P>;
  T* t = (T*)calloc(1, sizeof(T));
  if (!t) return CVWENO_ERR_NOMEM;
  cvweno_status st = fill_into<DIM, P>(t, m->dx, m->dy);
  if (st != CVWENO_OK) {
    free(t);
    return st;
  }
  m->tables = t;
  m->tables_bytes = sizeof(T);
  return CVWENO_OK;
}

// Gauss-Lobatto-Legendre nodes: the endpoints and the interior nodes, which are the
// zeros of P_p' (a multiple of the Jacobi polynomial P^(1,1)_{p-1}), obtained as the
// eigenvalues of the symmetric Jacobi matrix of the (1,1) recurrence with
// off-diagonal sqrt(k (k+2) / ((2k+1)(2k+3))).
void gll_nodes(int p, double* x) {
  x[0] = -1.0;
  x[p] = 1.0;
  const int n = p - 1;
  if (n <= 0) return;
  double J[kMaxEig][kMaxEig] = {}, lam[kMaxEig], V[kMaxEig][kMaxEig];
  for (int k = 1; k < n; ++k) {
    const double b = sqrt(k * (k + 2.0) / ((2.0 * k + 1.0) * (2.0 * k + 3.0)));
    J[k - 1][k] = J[k][k - 1] = b;
  }
  jacobi_eigen(n, J, lam, V);
  double srt[kMaxEig];
  for (int i = 0; i < n; ++i) srt[i] = lam[i];
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j)
      if (srt[j] < srt[i]) { double t = srt[i]; srt[i] = srt[j]; srt[j] = t; }
  for (int i = 0; i < n; ++i) x[i + 1] = srt[i];
}

// Lagrange basis on nodes x[0..p]: value and first derivative of l_a at y (product rule)
void lagrange_eval(int p, const double* x, int a, double y, double* val, double* der) {
  double v = 1.0, d = 0.0;
  for (int b = 0; b <= p; ++b) {
    if (b == a) continue;
    const double f = (y - x[b]) / (x[a] - x[b]);
    d = d * f + v / (x[a] - x[b]);
    v *= f;
  }
  *val = v;
  *der = d;
}

template <int DIM, int P>
cvweno_status fill_cg(cvweno_mesh m) {
  using C = CgTables<DIM, P>;
  constexpr int N = P + 1;
  C* t = (C*)calloc(1, sizeof(C));
  if (!t) return CVWENO_ERR_NOMEM;
  double xg[N], gx[N], gw[N];
  gll_nodes(P, xg);
  gauss_golub_welsch(N, gx, gw);
  const int NG = 8;
  double qx[NG], qw[NG];
  gauss_golub_welsch(NG, qx, qw);
  for (int a = 0; a < N; ++a) {
    t->xg[a] = (float)xg[a];
    m->cg_xg[a] = xg[a];
    for (int q = 0; q < N; ++q) {
      double v, d;
      lagrange_eval(P, xg, a, gx[q], &v, &d);
      t->Lq[q][a] = (float)v;
      t->Ldq[q][a] = (float)d;
    }
    double wl = 0.0;
    for (int q = 0; q < NG; ++q) {
      double va, da;
      lagrange_eval(P, xg, a, qx[q], &va, &da);
      wl += qw[q] * va;
    }
    t->wl[a] = (float)wl;
    t->iml[a] = (float)(1.0 / ((a == 0 ? 2.0 : 1.0) * wl));
    m->cg_wl[a] = wl;
  }
  // Em[a][m] = int l_a P_m, Dm[a][m] = int l_a P_m' (exact: degree <= 2p < 2 NG)
  for (int a = 0; a < N; ++a)
    for (int mm = 0; mm < N; ++mm) {
      double e = 0.0, dd = 0.0, tab[2 * N];
      for (int q = 0; q < NG; ++q) {
        double va, da;
        lagrange_eval(P, xg, a, qx[q], &va, &da);
        legendre_derivs(qx[q], P, 1, tab);
        e += qw[q] * va * tab[mm];
        dd += qw[q] * va * tab[N + mm];
      }
      t->Em[a][mm] = (float)e;
      t->Dm[a][mm] = (float)dd;
    }
  // V[m][a] = (2m+1)/2 int P_m l_a and M1[a][b] = int l_a l_b, in FP64 then rounded once
  for (int mm = 0; mm < N; ++mm)
    for (int a = 0; a < N; ++a) {
      double acc = 0.0, tab[N * N];
      for (int q = 0; q < NG; ++q) {
        double va, da;
        lagrange_eval(P, xg, a, qx[q], &va, &da);
        legendre_derivs(qx[q], P, 0, tab);
        acc += qw[q] * tab[mm] * va;
      }
      t->V[mm][a] = (float)(0.5 * (2 * mm + 1) * acc);
    }
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b) {
      double acc = 0.0;
      for (int q = 0; q < NG; ++q) {
        double va, da, vb, db;
        lagrange_eval(P, xg, a, qx[q], &va, &da);
        lagrange_eval(P, xg, b, qx[q], &vb, &db);
        acc += qw[q] * va * vb;
      }
      t->M1[a][b] = (float)acc;
    }
  m->cg_tables = t;
  m->cg_tables_bytes = sizeof(C);
  return CVWENO_OK;
}

}  // namespace

bool gauss_rule(int n, double* x, double* w) { return gauss_golub_welsch(n, x, w); }

cvweno_status fill_dg_tables(int dim, int p, double dx, double dy, void* out, size_t capacity, size_t* bytes) {
  switch (dim * 10 + p) {
#define CVW_FILL(D, Q)                                                               \
  case D * 10 + Q:                                                                   \
    if (capacity < sizeof(DgTables<D, Q>)) return CVWENO_ERR_ARG;                    \
    *bytes = sizeof(DgTables<D, Q>);                                                 \
    return fill_into<D, Q>(static_cast<DgTables<D, Q>*>(out), dx, dy);
    CVW_FILL(1, 1) CVW_FILL(1, 2) CVW_FILL(1, 3) CVW_FILL(1, 4)
    CVW_FILL(2, 1) CVW_FILL(2, 2) CVW_FILL(2, 3) CVW_FILL(2, 4)
#undef CVW_FILL
    default: return CVWENO_ERR_UNSUPPORTED;
  }
}

void legendre_values(double x, int mmax, double* out) { legendre_derivs(x, mmax, 0, out); }

cvweno_status build_tables(cvweno_mesh m) {
  // integer mesh tables
  const int nx = m->nx, ny = m->ny, nc = m->ncorner;
  const int perx = m->desc.bc[0] == CVWENO_PERIODIC, pery = m->dim == 2 && m->desc.bc[2] == CVWENO_PERIODIC;
  m->cell_vertices = (int32_t*)malloc(sizeof(int32_t) * m->ncell * nc);
  m->vertex_cells = (int32_t*)malloc(sizeof(int32_t) * m->nvert * nc);
  m->colour = (int32_t*)malloc(sizeof(int32_t) * m->ncell);
  if (!m->cell_vertices || !m->vertex_cells || !m->colour) return CVWENO_ERR_NOMEM;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      int64_t e = i + (int64_t)nx * j;
      for (int c = 0; c < nc; ++c) {
        int I = i + (c & 1), J = j + ((c >> 1) & 1);
        if (perx && I == nx) I = 0;
        if (pery && J == ny) J = 0;
        m->cell_vertices[e * nc + c] = (int32_t)(I + (int64_t)m->vx * J);
      }
      int cx = (perx && (nx & 1) && i == nx - 1) ? 2 : (i & 1);
      int cy = m->dim == 2 ? ((pery && (ny & 1) && j == ny - 1) ? 2 : (j & 1)) : 0;
      m->colour[e] = cx + 3 * cy;
    }
  for (int J = 0; J < m->vy; ++J)
    for (int I = 0; I < m->vx; ++I) {
      int64_t v = I + (int64_t)m->vx * J;
      for (int s = 0; s < nc; ++s) {
        int ci = I - 1 + (s & 1), cj = m->dim == 2 ? J - 1 + ((s >> 1) & 1) : 0;
        if (perx) ci = (ci + nx) % nx;
        if (pery) cj = (cj + ny) % ny;
        bool ok = ci >= 0 && ci < nx && cj >= 0 && cj < ny;
        m->vertex_cells[v * nc + s] = ok ? (int32_t)(ci + (int64_t)nx * cj) : -1;
      }
    }
  // reference tabulations
  cvweno_status st;
  switch (m->dim * 10 + m->p) {
    case 11: st = fill<1, 1>(m); if (st == CVWENO_OK && m->kind == CVWENO_CG) st = fill_cg<1, 1>(m); return st;
    case 12: st = fill<1, 2>(m); if (st == CVWENO_OK && m->kind == CVWENO_CG) st = fill_cg<1, 2>(m); return st;
    case 13: st = fill<1, 3>(m); if (st == CVWENO_OK && m->kind == CVWENO_CG) st = fill_cg<1, 3>(m); return st;
    case 14: st = fill<1, 4>(m); if (st == CVWENO_OK && m->kind == CVWENO_CG) st = fill_cg<1, 4>(m); return st;
    case 21: st = fill<2, 1>(m); if (st == CVWENO_OK && m->kind == CVWENO_CG) st = fill_cg<2, 1>(m); return st;
    case 22: st = fill<2, 2>(m); if (st == CVWENO_OK && m->kind == CVWENO_CG) st = fill_cg<2, 2>(m); return st;
    case 23: st = fill<2, 3>(m); if (st == CVWENO_OK && m->kind == CVWENO_CG) st = fill_cg<2, 3>(m); return st;
    case 24: st = fill<2, 4>(m); if (st == CVWENO_OK && m->kind == CVWENO_CG) st = fill_cg<2, 4>(m); return st;
    default: return CVWENO_ERR_UNSUPPORTED;
  }
}

}  // namespace cvw
