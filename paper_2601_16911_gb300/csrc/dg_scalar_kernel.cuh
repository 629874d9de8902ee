// Fused per-stage kernel for scalar conservation laws (DG, tensor Legendre Q_p).
//
// One CTA owns a TX x TY tile of cells.  It stages the tile plus a one-cell halo of
// Legendre coefficients in shared memory (coalesced row loads, transposed to a
// mode-major layout so that thread-per-cell reads are bank-conflict free), and then
// runs every stage of the path without touching HBM in between:
//
//   (a)+(b) vertex phase, one thread per tile vertex: Taylor data of the (up to)
//           four cells around the vertex at that vertex (eq. taylorsol), their
//           pointwise indicators (eq. pointsnorm), Jiang-Shu weights with equal linear
//           weights and the vertex candidate t* (eq. taylorcand), gathered in the fixed
//           slot order SW, SE, NW, NE -- no atomics, so results are deterministic;
//   (c)     cell phase, one thread per cell: the 2^d vertex candidates mapped into the
//           cell's semi-norm coordinates by precomputed corner matrices (Sec. 3.2
//           remark), Jiang-Shu cell weights, the reconstruction u*, the sensor
//           gamma_e (eq. gamma) and nu_e = lambda_e h_e / (2p) (eq. lostab);
//   (d)     in troubled cells (gamma_e < C_gamma): pointwise indicators at the Gauss
//           nodes and the dissipation-preserving weights alpha_q (eq. alphaq);
//   (e)     LLF face fluxes, the volume flux term and the alpha-weighted viscous term
//           by sum factorisation, M^{-1} (diagonal) and the SSP-RK3 stage combination
//           in the epilogue.  Fluxes are evaluated as deviations from the flux of the
//           cell mean (exact: a constant flux has zero residual), so FP32 rounding is
//           relative to the variation within a cell, not to |f(u)|.
//
// All arithmetic is FP32.  The tabulations arrive through a __grid_constant__ kernel
// parameter, so fully unrolled loops read them as constant-bank operands.
#pragma once

#include "cvweno_internal.cuh"

namespace cvw {

__device__ __forceinline__ float ipowf(float x, int r) {
  float y = x;
  for (int i = 1; i < r; ++i) y *= x;
  return y;
}

__device__ __forceinline__ float powq(float x, float q) { return q == 1.0f ? x : powf(x, q); }

// ---- scalar fluxes, evaluated as deviations from the cell mean -------------------------
// A law object is built per cell from its mean ubar.  flux_dev returns
// f(ubar + d) - f(ubar) in forms whose rounding is relative to |d|; llf_dev returns the
// LLF flux minus f(ubar) . n.  The constant f(ubar) cancels exactly between the volume
// and face terms of every test function, so it is never formed.
template <int SYS, int DIM>
struct ScalarLaw;

template <int DIM>
struct ScalarLaw<CVWENO_BURGERS, DIM> {
  float ubar;
  __device__ __forceinline__ ScalarLaw(const StageArgs&, float ub) : ubar(ub) {}
  __device__ __forceinline__ float dev(float d) const { return d * fmaf(0.5f, d, ubar); }
  __device__ __forceinline__ void flux_dev(float d, float& fx, float& fy) const {
    fx = dev(d);
    fy = fx;
  }
  __device__ __forceinline__ float flux_dev_dir(float d, int) const { return dev(d); }
  // |f'(u)| (Euclidean) for nu_e, and |f'(u) . n| for an axis-aligned face
  __device__ __forceinline__ float speed(float u) const { return DIM == 2 ? 1.41421356237f * fabsf(u) : fabsf(u); }
  __device__ __forceinline__ float nspeed(float u, int) const { return fabsf(u); }
};

template <int DIM>
struct ScalarLaw<CVWENO_KPP, DIM> {
  float sb, cb;  // sin(ubar), cos(ubar)
  __device__ __forceinline__ ScalarLaw(const StageArgs&, float ub) { sincosf(ub, &sb, &cb); }
  // sin(ub + d) - sin(ub) = sin(ub)(cos d - 1) + cos(ub) sin d, and likewise for cos;
  // cos d - 1 = -sin^2 d / (1 + cos d) avoids the cancellation where cos d > 0
  __device__ __forceinline__ void flux_dev(float d, float& fx, float& fy) const {
    float s, c;
    sincosf(d, &s, &c);
    const float cm1 = c > 0.0f ? -(s * s) / (1.0f + c) : c - 1.0f;
    fx = fmaf(sb, cm1, cb * s);
    fy = fmaf(cb, cm1, -sb * s);
  }
  __device__ __forceinline__ float flux_dev_dir(float d, int dir) const {
    float fx, fy;
    flux_dev(d, fx, fy);
    return dir == 0 ? fx : fy;
  }
  __device__ __forceinline__ float speed(float) const { return 1.0f; }
  __device__ __forceinline__ float nspeed(float u, int dir) const {
    return dir == 0 ? fabsf(cosf(u)) : fabsf(sinf(u));
  }
};

template <int DIM>
struct ScalarLaw<CVWENO_LINADV, DIM> {
  float vx, vy;
  __device__ __forceinline__ ScalarLaw(const StageArgs& a, float) : vx(a.adv_vx), vy(a.adv_vy) {}
  __device__ __forceinline__ void flux_dev(float d, float& fx, float& fy) const {
    fx = vx * d;
    fy = vy * d;
  }
  __device__ __forceinline__ float flux_dev_dir(float d, int dir) const { return (dir == 0 ? vx : vy) * d; }
  __device__ __forceinline__ float speed(float) const { return DIM == 2 ? sqrtf(vx * vx + vy * vy) : fabsf(vx); }
  __device__ __forceinline__ float nspeed(float, int dir) const { return fabsf(dir == 0 ? vx : vy); }
};

// LLF flux in direction dir (0 = x, 1 = y) minus f(ubar) . n, from the left/lower
// state ubar + dL to the right/upper state ubar + dR (reading A14).
template <class Law>
__device__ __forceinline__ float llf_dev(const Law& law, const StageArgs& a, float ubar, float dL, float dR, int dir) {
  const float lam = a.lambda_const > 0.0f ? a.lambda_const
                                          : fmaxf(law.nspeed(ubar + dL, dir), law.nspeed(ubar + dR, dir));
  return 0.5f * (law.flux_dev_dir(dL, dir) + law.flux_dev_dir(dR, dir)) - 0.5f * lam * (dR - dL);
}

// Reference Taylor data t[k] = d^k u (s_x, s_y) at corner (SX, SY) of one cell whose
// coefficients sit at c[m * stride].
template <int DIM, int P, int SX, int SY>
__device__ __forceinline__ void corner_taylor(const DgTables<DIM, P>& T, const float* c, int stride, float* t) {
  constexpr int N = P + 1;
  if constexpr (DIM == 1) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      float acc = 0.0f;
#pragma unroll
      for (int m = 0; m < N; ++m) {
        float e = (SX < 0 && ((m + k) & 1)) ? -T.E[k][m] : T.E[k][m];
        acc = fmaf(e, c[m * stride], acc);
      }
      t[k] = acc;
    }
  } else {
    float cl[N * N];
#pragma unroll
    for (int m = 0; m < N * N; ++m) cl[m] = c[m * stride];
    float tmp[N][N];  // [kx][my]
#pragma unroll
    for (int kx = 0; kx < N; ++kx)
#pragma unroll
      for (int my = 0; my < N; ++my) {
        float acc = 0.0f;
#pragma unroll
        for (int mx = 0; mx < N; ++mx) {
          float e = (SX < 0 && ((mx + kx) & 1)) ? -T.E[kx][mx] : T.E[kx][mx];
          acc = fmaf(e, cl[mx + N * my], acc);
        }
        tmp[kx][my] = acc;
      }
#pragma unroll
    for (int ky = 0; ky < N; ++ky)
#pragma unroll
      for (int kx = 0; kx < N; ++kx) {
        float acc = 0.0f;
#pragma unroll
        for (int my = 0; my < N; ++my) {
          float e = (SY < 0 && ((my + ky) & 1)) ? -T.E[ky][my] : T.E[ky][my];
          acc = fmaf(e, tmp[kx][my], acc);
        }
        t[kx + N * ky] = acc;
      }
  }
}

// One slot of the vertex gather: cell at halo (hx, hy), touching corner (SX, SY).
template <int DIM, int P, int SX, int SY>
__device__ __forceinline__ void vertex_slot(const StageArgs& a, const DgTables<DIM, P>& T, const float* cell, int stride,
                                            float* acc, float& wsum) {
  constexpr int ND = DgTables<DIM, P>::ND;
  float t[ND];
  corner_taylor<DIM, P, SX, SY>(T, cell, stride, t);
  float b2 = 0.0f;
#pragma unroll
  for (int k = 1; k < ND; ++k) b2 = fmaf(T.sigma[k] * t[k], t[k], b2);
  float beta = powq(sqrtf(b2), a.q);
  float wt = 1.0f / ipowf(a.eps + beta, a.r);
  wsum += wt;
#pragma unroll
  for (int k = 0; k < ND; ++k) acc[k] = fmaf(wt, t[k], acc[k]);
}

template <int DIM, int P, int SYS, int TX, int TY>
__global__ void __launch_bounds__(TX* TY)
    dg_scalar_stage(const __grid_constant__ StageArgs a, const __grid_constant__ DgTables<DIM, P> T) {
  using Tb = DgTables<DIM, P>;
  using Law = ScalarLaw<SYS, DIM>;
  constexpr int N = P + 1, ND = Tb::ND, NS = Tb::NS, NC = Tb::NC;
  constexpr int NT = TX * TY;
  constexpr int HX = TX + 2, HY = DIM == 2 ? TY + 2 : 1, NH = HX * HY;
  constexpr int VXT = TX + 1, VYT = DIM == 2 ? TY + 1 : 1, NVT = VXT * VYT;
  extern __shared__ float smem[];
  float* sc = smem;           // [ND][NH]  coefficients, mode-major
  float* st = smem + ND * NH; // [ND][NVT] vertex candidates t* (reference units)

  const int nx = a.nx, ny = DIM == 2 ? a.ny : 1;
  const int i0 = blockIdx.x * TX, j0 = DIM == 2 ? blockIdx.y * TY : 0;

  // ---- load tile + halo ------------------------------------------------------------
  for (int f = threadIdx.x; f < NH * ND; f += NT) {
    int r = f / (HX * ND);
    int rem = f - r * (HX * ND);
    int cc = rem / ND;
    int mm = rem - cc * ND;
    int gi = i0 - 1 + cc, gj = DIM == 2 ? j0 - 1 + r : 0;
    bool ok = true;
    if (gi < 0 || gi >= nx) {
      if (a.perx) gi = (gi + nx) % nx; else ok = false;
    }
    if (DIM == 2 && (gj < 0 || gj >= ny)) {
      if (a.pery) gj = (gj + ny) % ny; else ok = false;
    }
    sc[mm * NH + r * HX + cc] = ok ? __ldg(a.u_in + ((size_t)gj * nx + gi) * ND + mm) : 0.0f;
  }
  __syncthreads();

  // ---- (a)+(b): vertex candidates of the tile's vertices ------------------------------
  const int act_x = min(TX, nx - i0), act_y = DIM == 2 ? min(TY, ny - j0) : 1;
  for (int v = threadIdx.x; v < NVT; v += NT) {
    int va = v % VXT, vb = DIM == 2 ? v / VXT : 0;
    if (va > act_x || (DIM == 2 && vb > act_y)) continue;
    float acc[ND];
#pragma unroll
    for (int k = 0; k < ND; ++k) acc[k] = 0.0f;
    float wsum = 0.0f;
    // halo coordinates of the SW (1D: W) cell of this vertex
    const int gi_w = i0 - 1 + va, gj_s = j0 - 1 + vb;
    const bool has_w = a.perx || gi_w >= 0, has_e = a.perx || gi_w + 1 < nx;
    const bool has_s = DIM == 1 || a.pery || gj_s >= 0, has_n = DIM == 1 || a.pery || gj_s + 1 < ny;
    const float* base = sc + (DIM == 2 ? vb * HX : 0) + va;
    if constexpr (DIM == 1) {
      if (has_w) vertex_slot<1, P, 1, 1>(a, T, base, NH, acc, wsum);
      if (has_e) vertex_slot<1, P, -1, 1>(a, T, base + 1, NH, acc, wsum);
    } else {
      if (has_w && has_s) vertex_slot<2, P, 1, 1>(a, T, base, NH, acc, wsum);
      if (has_e && has_s) vertex_slot<2, P, -1, 1>(a, T, base + 1, NH, acc, wsum);
      if (has_w && has_n) vertex_slot<2, P, 1, -1>(a, T, base + HX, NH, acc, wsum);
      if (has_e && has_n) vertex_slot<2, P, -1, -1>(a, T, base + HX + 1, NH, acc, wsum);
    }
    const float inv = 1.0f / wsum;
#pragma unroll
    for (int k = 0; k < ND; ++k) st[k * NVT + v] = acc[k] * inv;
    if (a.tstar_out) {
      int I = i0 + va, J = j0 + vb;
      bool own_x = (va < TX || I == nx) && I < a.vx;
      int vyn = DIM == 2 ? (a.pery ? ny : ny + 1) : 1;
      bool own_y = DIM == 1 || ((vb < TY || J == ny) && J < vyn);
      if (own_x && own_y) {
        size_t vi = (size_t)I + (size_t)a.vx * J;
#pragma unroll
        for (int k = 0; k < ND; ++k) a.tstar_out[vi * ND + k] = acc[k] * inv * T.tscale[k];
      }
    }
  }
  __syncthreads();

  // ---- one thread per cell from here on (no further barriers) ----------------------------
  const int tx = threadIdx.x % TX, ty = DIM == 2 ? threadIdx.x / TX : 0;
  const int gi = i0 + tx, gj = j0 + ty;
  if (gi >= nx || gj >= ny) return;
  const int hc = (DIM == 2 ? (ty + 1) * HX : 0) + tx + 1;
  const size_t cell = (size_t)gj * nx + gi;
  float c[ND];
#pragma unroll
  for (int m = 0; m < ND; ++m) c[m] = sc[m * NH + hc];

  // ---- (c) cell-vertex reconstruction and sensor --------------------------------------
  float w0[NS];
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    float acc = 0.0f;
#pragma unroll
    for (int j = i; j < NS; ++j) acc = fmaf(T.R[i][j], c[j + 1], acc);
    w0[i] = acc;
  }
  float n0sq = 0.0f;
#pragma unroll
  for (int i = 0; i < NS; ++i) n0sq = fmaf(w0[i], w0[i], n0sq);
  const float n0 = sqrtf(n0sq);
  float gam;
  {
    const float om0 = (1.0f - NC * a.gamma_vertex) / ipowf(a.eps + powq(n0, a.q), a.r);
    float S[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) S[i] = om0 * w0[i];
    float osum = om0;
#pragma unroll
    for (int l = 0; l < NC; ++l) {
      const int vi = (tx + (l & 1)) + (DIM == 2 ? (ty + ((l >> 1) & 1)) * VXT : 0);
      float tl[NS];
#pragma unroll
      for (int k = 0; k < NS; ++k) tl[k] = st[(k + 1) * NVT + vi];
      float wl[NS];
      float b2 = 0.0f;
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        float acc = 0.0f;
#pragma unroll
        for (int j = 0; j < NS; ++j) acc = fmaf(T.A[l][i][j], tl[j], acc);
        wl[i] = acc;
        b2 = fmaf(acc, acc, b2);
      }
      const float om = a.gamma_vertex / ipowf(a.eps + powq(sqrtf(b2), a.q), a.r);
      osum += om;
#pragma unroll
      for (int i = 0; i < NS; ++i) S[i] = fmaf(om, wl[i], S[i]);
    }
    const float inv = 1.0f / osum;
    float d2 = 0.0f;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      float df = w0[i] - S[i] * inv;
      d2 = fmaf(df, df, d2);
    }
    if (a.sensor_mode == CVWENO_SENSOR_SMOOTH)
      gam = 1.0f;
    else if (a.sensor_mode == CVWENO_SENSOR_TROUBLED)
      gam = 0.0f;
    else if (n0 <= 1e-30f)
      gam = 1.0f;
    else
      gam = 1.0f - powq(fminf(1.0f, sqrtf(d2) / n0), a.q);
  }

  // ---- values at volume Gauss nodes, in deviation form -------------------------------------
  // u(x_q) = ubar + dU[q] with dU built from the non-mean modes only, so rounding is
  // relative to the variation inside the cell rather than to |u| (the mean cancels
  // exactly between the volume and face terms of every mode).
  const float ubar = c[0];
  const Law law(a, ubar);
  float cz[ND];
#pragma unroll
  for (int m = 0; m < ND; ++m) cz[m] = m == 0 ? 0.0f : c[m];
  float dU[ND], Ux[ND], Uy[ND];
  if constexpr (DIM == 1) {
#pragma unroll
    for (int q = 0; q < N; ++q) {
      float u = 0.0f, ux = 0.0f;
#pragma unroll
      for (int m = 1; m < N; ++m) {
        u = fmaf(T.B[q][m], cz[m], u);
        ux = fmaf(T.Bd[q][m], cz[m], ux);
      }
      dU[q] = u;
      Ux[q] = ux;
      Uy[q] = 0.0f;
    }
  } else {
#pragma unroll
    for (int qx = 0; qx < N; ++qx) {
      float tb[N], td[N];
#pragma unroll
      for (int my = 0; my < N; ++my) {
        float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
        for (int mx = 0; mx < N; ++mx) {
          s0 = fmaf(T.B[qx][mx], cz[mx + N * my], s0);
          s1 = fmaf(T.Bd[qx][mx], cz[mx + N * my], s1);
        }
        tb[my] = s0;
        td[my] = s1;
      }
#pragma unroll
      for (int qy = 0; qy < N; ++qy) {
        float u = 0.0f, ux = 0.0f, uy = 0.0f;
#pragma unroll
        for (int my = 0; my < N; ++my) {
          u = fmaf(T.B[qy][my], tb[my], u);
          ux = fmaf(T.B[qy][my], td[my], ux);
          uy = fmaf(T.Bd[qy][my], tb[my], uy);
        }
        dU[qx + N * qy] = u;
        Ux[qx + N * qy] = ux;
        Uy[qx + N * qy] = uy;
      }
    }
  }

  // ---- own traces at the face Gauss nodes (deviations from ubar) ------------------------
  // 1D: one node per face.  2D: x-faces carry N nodes in eta, y-faces N nodes in xi.
  constexpr int NF = DIM == 2 ? N : 1;
  float oR[NF], oL[NF], oT[NF], oB[NF];
  {
    if constexpr (DIM == 1) {
      float sR = 0.0f, sL = 0.0f;
#pragma unroll
      for (int m = 1; m < N; ++m) {
        sR += cz[m];
        sL += (m & 1) ? -cz[m] : cz[m];
      }
      oR[0] = sR;
      oL[0] = sL;
    } else {
      float trR[N], trL[N], trT[N], trB[N];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        float r = 0.0f, l = 0.0f, t = 0.0f, b = 0.0f;
#pragma unroll
        for (int i = 0; i < N; ++i) {
          r += cz[i + N * j];
          l += (i & 1) ? -cz[i + N * j] : cz[i + N * j];
          t += cz[j + N * i];
          b += (i & 1) ? -cz[j + N * i] : cz[j + N * i];
        }
        trR[j] = r;
        trL[j] = l;
        trT[j] = t;
        trB[j] = b;
      }
#pragma unroll
      for (int q = 0; q < N; ++q) {
        float r = 0.0f, l = 0.0f, t = 0.0f, b = 0.0f;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          r = fmaf(T.B[q][j], trR[j], r);
          l = fmaf(T.B[q][j], trL[j], l);
          t = fmaf(T.B[q][j], trT[j], t);
          b = fmaf(T.B[q][j], trB[j], b);
        }
        oR[q] = r;
        oL[q] = l;
        oT[q] = t;
        oB[q] = b;
      }
    }
  }

  // ---- lambda_e, nu_e ---------------------------------------------------------------------
  float lam;
  if (a.lambda_const > 0.0f) {
    lam = a.lambda_const;
  } else {
    lam = 0.0f;
#pragma unroll
    for (int q = 0; q < ND; ++q) lam = fmaxf(lam, law.speed(ubar + dU[q]));
#pragma unroll
    for (int q = 0; q < NF; ++q) {
      lam = fmaxf(lam, law.speed(ubar + oR[q]));
      lam = fmaxf(lam, law.speed(ubar + oL[q]));
      if constexpr (DIM == 2) {
        lam = fmaxf(lam, law.speed(ubar + oT[q]));
        lam = fmaxf(lam, law.speed(ubar + oB[q]));
      }
    }
  }
  const float nu = lam * a.nu_scale;
  if (a.gamma_out) a.gamma_out[cell] = gam;
  if (a.nu_out) a.nu_out[cell] = nu;
  if (a.lambda_out) a.lambda_out[cell] = lam;
  if (a.mode & kModeSensorOnly) return;

  // ---- (d) shock-capturing quadrature weights ---------------------------------------------
  bool troubled = a.sc && gam < a.c_gamma && n0 > 1e-30f;
  if (a.troubled_override) {
    int ov = a.troubled_override[cell];
    if (ov >= 0) troubled = ov && n0 > 1e-30f;
  }
  float alpha[ND];
#pragma unroll
  for (int q = 0; q < ND; ++q) alpha[q] = 1.0f;
  if (troubled && gam < 1.0f) {
    float Nq[ND];
    if constexpr (DIM == 1) {
#pragma unroll
      for (int q = 0; q < N; ++q) {
        float s2 = 0.0f;
#pragma unroll
        for (int k = 1; k < N; ++k) {
          float d = 0.0f;
#pragma unroll
          for (int m = 0; m < N; ++m) d = fmaf(T.Bk[k][q][m], c[m], d);
          s2 = fmaf(T.sigma[k] * d, d, s2);
        }
        Nq[q] = sqrtf(s2);
      }
    } else {
#pragma unroll
      for (int qx = 0; qx < N; ++qx) {
        float X[N][N];  // [kx][my]
#pragma unroll
        for (int kx = 0; kx < N; ++kx)
#pragma unroll
          for (int my = 0; my < N; ++my) {
            float acc = 0.0f;
#pragma unroll
            for (int mx = 0; mx < N; ++mx) acc = fmaf(T.Bk[kx][qx][mx], c[mx + N * my], acc);
            X[kx][my] = acc;
          }
#pragma unroll
        for (int qy = 0; qy < N; ++qy) {
          float s2 = 0.0f;
#pragma unroll
          for (int ky = 0; ky < N; ++ky)
#pragma unroll
            for (int kx = 0; kx < N; ++kx) {
              if (kx + ky == 0) continue;
              float d = 0.0f;
#pragma unroll
              for (int my = 0; my < N; ++my) d = fmaf(T.Bk[ky][qy][my], X[kx][my], d);
              s2 = fmaf(T.sigma[kx + N * ky] * d, d, s2);
            }
          Nq[qx + N * qy] = sqrtf(s2);
        }
      }
    }
    float s1 = 0.0f, s2 = 0.0f;
#pragma unroll
    for (int q = 0; q < ND; ++q) {
      const int qx = q % N, qy = q / N;
      const float W = DIM == 2 ? T.w[qx] * T.w[qy] : T.w[q];
      float gx = a.two_dx * Ux[q], gy = a.two_dy * Uy[q];
      float g = fmaf(gx, gx, DIM == 2 ? gy * gy : 0.0f);
      s1 = fmaf(W, g, s1);
      s2 = fmaf(W * Nq[q], g, s2);
    }
    if (s2 > 0.0f) {
      const float f = s1 / s2;
#pragma unroll
      for (int q = 0; q < ND; ++q) alpha[q] = Nq[q] * f;
    }
  }
  if (a.troubled_out) a.troubled_out[cell] = troubled ? 1 : 0;
  if (a.alpha_out) {
#pragma unroll
    for (int q = 0; q < ND; ++q) a.alpha_out[cell * ND + q] = alpha[q];
  }

  // ---- (e) residual, deviation form ----------------------------------------------------------
  float r[ND];
#pragma unroll
  for (int m = 0; m < ND; ++m) r[m] = 0.0f;
  const float mu = (1.0f - gam) * nu;
  // faces: neighbour traces relative to this cell's mean (ghost = own trace on a
  // transmissive side)
  {
    const bool hasR = a.perx || gi + 1 < nx, hasL = a.perx || gi > 0;
    float FR[NF], FL[NF];
    if constexpr (DIM == 1) {
      float nbR = oR[0], nbL = oL[0];
      if (hasR) {
        float s = 0.0f;
#pragma unroll
        for (int m = 1; m < N; ++m) s += (m & 1) ? -sc[m * NH + hc + 1] : sc[m * NH + hc + 1];
        nbR = (sc[hc + 1] - ubar) + s;
      }
      if (hasL) {
        float s = 0.0f;
#pragma unroll
        for (int m = 1; m < N; ++m) s += sc[m * NH + hc - 1];
        nbL = (sc[hc - 1] - ubar) + s;
      }
      FR[0] = llf_dev(law, a, ubar, oR[0], nbR, 0);
      FL[0] = llf_dev(law, a, ubar, nbL, oL[0], 0);
#pragma unroll
      for (int m = 0; m < N; ++m) r[m] = -a.two_dx * (FR[0] - ((m & 1) ? -FL[0] : FL[0]));
    } else {
      const bool hasT = a.pery || gj + 1 < ny, hasB = a.pery || gj > 0;
      float FT[NF], FB[NF];
      float nR[N], nL[N], nT[N], nB[N];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        float r0 = 0.0f, l0 = 0.0f, t0 = 0.0f, b0 = 0.0f;
#pragma unroll
        for (int i = 0; i < N; ++i) {
          // right neighbour's left trace (xi = -1), left neighbour's right trace (xi = +1),
          // top neighbour's bottom trace (eta = -1), bottom neighbour's top trace (eta = +1);
          // the neighbours' means are added after the projection onto the face nodes
          const int mr = i + N * j, mt = j + N * i;
          if (mr != 0) {
            float cr = sc[mr * NH + hc + 1], cl = sc[mr * NH + hc - 1];
            r0 += (i & 1) ? -cr : cr;
            l0 += cl;
          }
          if (mt != 0) {
            float ct = sc[mt * NH + hc + HX], cb = sc[mt * NH + hc - HX];
            t0 += (i & 1) ? -ct : ct;
            b0 += cb;
          }
        }
        nR[j] = r0;
        nL[j] = l0;
        nT[j] = t0;
        nB[j] = b0;
      }
      const float mR = sc[hc + 1] - ubar, mL = sc[hc - 1] - ubar;
      const float mT = sc[hc + HX] - ubar, mB = sc[hc - HX] - ubar;
#pragma unroll
      for (int q = 0; q < N; ++q) {
        float vr = 0.0f, vl = 0.0f, vt = 0.0f, vb = 0.0f;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          vr = fmaf(T.B[q][j], nR[j], vr);
          vl = fmaf(T.B[q][j], nL[j], vl);
          vt = fmaf(T.B[q][j], nT[j], vt);
          vb = fmaf(T.B[q][j], nB[j], vb);
        }
        vr = hasR ? mR + vr : oR[q];
        vl = hasL ? mL + vl : oL[q];
        vt = hasT ? mT + vt : oT[q];
        vb = hasB ? mB + vb : oB[q];
        FR[q] = llf_dev(law, a, ubar, oR[q], vr, 0);
        FL[q] = llf_dev(law, a, ubar, vl, oL[q], 0);
        FT[q] = llf_dev(law, a, ubar, oT[q], vt, 1);
        FB[q] = llf_dev(law, a, ubar, vb, oB[q], 1);
      }
      // project the face fluxes: r[mx,my] -= 2/dx (hR[my] - (-1)^mx hL[my]) + 2/dy (...)
      float hR[N], hL[N], hT[N], hB[N];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
#pragma unroll
        for (int q = 0; q < N; ++q) {
          float wb = T.w[q] * T.B[q][j];
          s0 = fmaf(wb, FR[q], s0);
          s1 = fmaf(wb, FL[q], s1);
          s2 = fmaf(wb, FT[q], s2);
          s3 = fmaf(wb, FB[q], s3);
        }
        hR[j] = s0;
        hL[j] = s1;
        hT[j] = s2;
        hB[j] = s3;
      }
#pragma unroll
      for (int my = 0; my < N; ++my)
#pragma unroll
        for (int mx = 0; mx < N; ++mx) {
          float fxv = hR[my] - ((mx & 1) ? -hL[my] : hL[my]);
          float fyv = hT[mx] - ((my & 1) ? -hB[mx] : hB[mx]);
          r[mx + N * my] = -(a.two_dx * fxv + a.two_dy * fyv);
        }
    }
  }
  // volume: flux deviation and alpha-weighted viscous term, projected by sum factorisation
  if constexpr (DIM == 1) {
#pragma unroll
    for (int q = 0; q < N; ++q) {
      float fx, fy;
      law.flux_dev(dU[q], fx, fy);
      float G = T.w[q] * (fx - mu * alpha[q] * a.two_dx * Ux[q]);
#pragma unroll
      for (int m = 1; m < N; ++m) r[m] = fmaf(a.two_dx * T.Bd[q][m], G, r[m]);
    }
  } else {
#pragma unroll
    for (int qx = 0; qx < N; ++qx) {
      float Gx[N], Gy[N];
#pragma unroll
      for (int qy = 0; qy < N; ++qy) {
        const int q = qx + N * qy;
        float fx, fy;
        law.flux_dev(dU[q], fx, fy);
        const float W = T.w[qx] * T.w[qy];
        Gx[qy] = W * (fx - mu * alpha[q] * a.two_dx * Ux[q]);
        Gy[qy] = W * (fy - mu * alpha[q] * a.two_dy * Uy[q]);
      }
      float hx[N], hy[N];
#pragma unroll
      for (int my = 0; my < N; ++my) {
        float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
        for (int qy = 0; qy < N; ++qy) {
          s0 = fmaf(T.B[qy][my], Gx[qy], s0);
          s1 = fmaf(T.Bd[qy][my], Gy[qy], s1);
        }
        hx[my] = s0;
        hy[my] = s1;
      }
#pragma unroll
      for (int my = 0; my < N; ++my)
#pragma unroll
        for (int mx = 0; mx < N; ++mx) {
          if (mx + my == 0) continue;
          float v = r[mx + N * my];
          v = fmaf(a.two_dx * T.Bd[qx][mx], hx[my], v);
          v = fmaf(a.two_dy * T.B[qx][mx], hy[my], v);
          r[mx + N * my] = v;
        }
    }
  }
  // M^{-1} and output
  bool bad = false;
  float* out = a.u_out + cell * ND;
  const float* un = a.u_n + cell * ND;
#pragma unroll
  for (int m = 0; m < ND; ++m) {
    const int mx = m % N, my = DIM == 2 ? m / N : 0;
    const float minv = DIM == 2 ? 0.25f * (2 * mx + 1) * (2 * my + 1) : 0.5f * (2 * mx + 1);
    float d = r[m] * minv;
    bad |= !isfinite(d);
    if (a.mode & kModeRK) {
      float v = a.rk_b * fmaf(a.dt, d, c[m]);
      if (a.rk_a != 0.0f) v = fmaf(a.rk_a, un[m], v);  // plain load: u_n may alias u_out
      out[m] = v;
    } else {
      out[m] = d;
    }
  }
  if (bad) atomicOr(a.status, kStatNonfinite);
}

}  // namespace cvw
