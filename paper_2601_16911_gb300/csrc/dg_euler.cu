// Fused stage kernel for the 2D compressible Euler equations (ideal gas), DG Q_p.
//
// Same tile structure as the scalar kernel: a TX x TY tile of cells plus a one-cell
// halo of all four conserved variables is staged in shared memory (mode-major), then
//   (a)+(b) vertex candidates of the density (Sec. 5.4: the sensor is computed from
//           the density and applied to all variables), one thread per tile vertex;
//   (c)     cell-vertex sensor gamma_e and nu_e = lambda_e h_e / (2p) with
//           lambda_e = max(|v| + c) over the cell's volume and face Gauss nodes;
//   (d)     SC weights: alpha~_q from the density's pointwise indicator, the
//           dissipation f_q of each conserved variable redistributed separately, so
//           each variable keeps its own cell dissipation rate (eq. alphaq);
//   (e)     HLL face fluxes with Davis wave-speed estimates, the volume flux and the
//           viscous term by sum factorisation, M^{-1}, and the SSP-RK3 combination.
//           As in the scalar kernel, every flux is evaluated as its deviation from the
//           flux of the cell's mean state (exact: a constant flux has zero residual),
//           so FP32 rounding is relative to the variation inside the cell.
// Non-positive density or pressure at any node raises the positivity bit of the
// status word (the computation continues; nothing traps).
#include "dg_scalar_kernel.cuh"

namespace cvw {
namespace {

constexpr int NV = 4;

// Mean state of a cell and the derived quantities the deviation fluxes need.
struct EulerMean {
  float U[NV];      // rho, m_x, m_y, E of the cell mean
  float vx, vy, H;  // mean velocity, E + p of the mean state
};

__device__ __forceinline__ EulerMean euler_mean(float g, const float* Ub) {
  EulerMean M;
#pragma unroll
  for (int v = 0; v < NV; ++v) M.U[v] = Ub[v];
  const float ir = 1.0f / Ub[0];
  M.vx = Ub[1] * ir;
  M.vy = Ub[2] * ir;
  const float p = (g - 1.0f) * (Ub[3] - 0.5f * (Ub[1] * M.vx + Ub[2] * M.vy));
  M.H = Ub[3] + p;
  return M;
}

// a*b - c*d with the rounding of c*d compensated (Kahan's FMA form): the result is
// accurate relative to itself even when the two products nearly cancel.
__device__ __forceinline__ float diff_of_products(float a, float b, float c, float d) {
  const float w = c * d;
  const float e = fmaf(-c, d, w);  // w - c*d, exactly
  const float f = fmaf(a, b, -w);  // a*b - w, one rounding
  return f + e;
}

// F(Ubar + d) - F(Ubar) in x and y, written as sums of (mean quantity) x (deviation)
// so that FP32 rounding is relative to |d|:
//   dv = (dm rhobar - mbar drho) / (rho rhobar),
//   dE - dK = (dE rhobar - dm . mbar / 2) / rhobar - (mbar + dm) . dv / 2,
//   dp = (g - 1)(dE - dK),  dH = dE + dp.
// The two differences that cancel exactly in uniform flow (dv for a uniform velocity,
// dE - dK for a uniform pressure) are formed with compensated products.
__device__ __forceinline__ void euler_dflux(float g, const EulerMean& M, const float* d, float* dFx, float* dFy) {
  const float rb = M.U[0];
  const float ir = 1.0f / (rb * (rb + d[0]));
  const float dvx = diff_of_products(d[1], rb, M.U[1], d[0]) * ir;
  const float dvy = diff_of_products(d[2], rb, M.U[2], d[0]) * ir;
  // dE rhobar - (dmx mbarx + dmy mbary) / 2, compensated
  const float x1 = diff_of_products(d[3], rb, 0.5f * d[1], M.U[1]);
  const float p2 = 0.5f * d[2] * M.U[2];
  const float e2 = fmaf(0.5f * d[2], M.U[2], -p2);
  const float x = (x1 - p2) - e2;
  const float dEmK = x / rb - 0.5f * ((M.U[1] + d[1]) * dvx + (M.U[2] + d[2]) * dvy);
  const float dp = (g - 1.0f) * dEmK;
  const float dH = d[3] + dp;
  dFx[0] = d[1];
  dFx[1] = M.U[1] * dvx + d[1] * M.vx + d[1] * dvx + dp;
  dFx[2] = M.U[2] * dvx + d[2] * M.vx + d[2] * dvx;
  dFx[3] = M.H * dvx + dH * M.vx + dH * dvx;
  dFy[0] = d[2];
  dFy[1] = M.U[1] * dvy + d[1] * M.vy + d[1] * dvy;
  dFy[2] = M.U[2] * dvy + d[2] * M.vy + d[2] * dvy + dp;
  dFy[3] = M.H * dvy + dH * M.vy + dH * dvy;
}

__device__ __forceinline__ float euler_pressure(float g, const float* U) {
  return (g - 1.0f) * (U[3] - 0.5f * (U[1] * U[1] + U[2] * U[2]) / U[0]);
}

// |v| + c at a node of full state U; flags non-positive density or pressure
__device__ __forceinline__ float euler_speed(float g, const float* U, bool& bad) {
  const float rho = U[0], ir = 1.0f / rho;
  const float vx = U[1] * ir, vy = U[2] * ir;
  const float p = euler_pressure(g, U);
  bad |= !(rho > 0.0f) || !(p > 0.0f);
  return sqrtf(vx * vx + vy * vy) + sqrtf(g * fmaxf(p, 0.0f) * fabsf(ir));
}

// HLL flux minus F(Ubar) . n across a face with normal +x (dir 0) or +y (dir 1), from
// the left/lower state Ubar + dL to the right/upper state Ubar + dR (reading A14, Davis
// wave speeds from the full states).  The constant F(Ubar) drops out of every branch:
// (S_R F(Ubar) - S_L F(Ubar)) / (S_R - S_L) = F(Ubar).
__device__ __forceinline__ void hll_dev(float g, const EulerMean& M, const float* dL, const float* dR, int dir, float* F,
                                        bool& bad) {
  float UL[NV], UR[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    UL[v] = M.U[v] + dL[v];
    UR[v] = M.U[v] + dR[v];
  }
  const float pL = euler_pressure(g, UL), pR = euler_pressure(g, UR);
  bad |= !(UL[0] > 0.0f) || !(UR[0] > 0.0f) || !(pL > 0.0f) || !(pR > 0.0f);
  const float vnl = UL[1 + dir] / UL[0], vnr = UR[1 + dir] / UR[0];
  const float cl = sqrtf(g * fmaxf(pL, 0.0f) / fabsf(UL[0])), cr = sqrtf(g * fmaxf(pR, 0.0f) / fabsf(UR[0]));
  const float sl = fminf(vnl - cl, vnr - cr), sr = fmaxf(vnl + cl, vnr + cr);
  float fxl[NV], fyl[NV], fxr[NV], fyr[NV];
  euler_dflux(g, M, dL, fxl, fyl);
  euler_dflux(g, M, dR, fxr, fyr);
  const float* fl = dir == 0 ? fxl : fyl;
  const float* fr = dir == 0 ? fxr : fyr;
  if (sl >= 0.0f) {
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = fl[v];
  } else if (sr <= 0.0f) {
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = fr[v];
  } else {
    const float inv = 1.0f / (sr - sl);
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = (sr * fl[v] - sl * fr[v] + sl * sr * (dR[v] - dL[v])) * inv;
  }
}

template <int P, int TX, int TY>
__global__ void __launch_bounds__(TX* TY)
    dg_euler_stage(const __grid_constant__ StageArgs a, const __grid_constant__ DgTables<2, P> T) {
  using Tb = DgTables<2, P>;
  constexpr int N = P + 1, ND = Tb::ND, NS = Tb::NS, NC = 4;
  constexpr int NT = TX * TY;
  constexpr int HX = TX + 2, HY = TY + 2, NH = HX * HY;
  constexpr int VXT = TX + 1, VYT = TY + 1, NVT = VXT * VYT;
  extern __shared__ float smem[];
  float* sc = smem;                 // [NV][ND][NH]
  float* st = smem + NV * ND * NH;  // [ND][NVT] density vertex candidates
  const int nx = a.nx, ny = a.ny;
  const size_t ncell = (size_t)nx * ny;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const float g = a.gas_gamma;

  // ---- load tile + halo of all variables ------------------------------------------------
  for (int f = threadIdx.x; f < NV * NH * ND; f += NT) {
    int v = f / (NH * ND);
    int rem0 = f - v * (NH * ND);
    int r = rem0 / (HX * ND);
    int rem = rem0 - r * (HX * ND);
    int cc = rem / ND;
    int mm = rem - cc * ND;
    int gi = i0 - 1 + cc, gj = j0 - 1 + r;
    bool ok = true;
    if (gi < 0 || gi >= nx) {
      if (a.perx) gi = (gi + nx) % nx; else ok = false;
    }
    if (gj < 0 || gj >= ny) {
      if (a.pery) gj = (gj + ny) % ny; else ok = false;
    }
    sc[(v * ND + mm) * NH + r * HX + cc] =
        ok ? __ldg(a.u_in + ((size_t)v * ncell + (size_t)gj * nx + gi) * ND + mm) : 0.0f;
  }
  __syncthreads();

  // ---- (a)+(b): density vertex candidates ---------------------------------------------------
  const int act_x = min(TX, nx - i0), act_y = min(TY, ny - j0);
  for (int vtx = threadIdx.x; vtx < NVT; vtx += NT) {
    int va = vtx % VXT, vb = vtx / VXT;
    if (va > act_x || vb > act_y) continue;
    float acc[ND];
#pragma unroll
    for (int k = 0; k < ND; ++k) acc[k] = 0.0f;
    float wsum = 0.0f;
    const int gi_w = i0 - 1 + va, gj_s = j0 - 1 + vb;
    const bool has_w = a.perx || gi_w >= 0, has_e = a.perx || gi_w + 1 < nx;
    const bool has_s = a.pery || gj_s >= 0, has_n = a.pery || gj_s + 1 < ny;
    const float* base = sc + vb * HX + va;
    // slots SW, SE, NW, NE (density block only)
#pragma unroll 1
    for (int s = 0; s < NC; ++s) {
      const int ex = s & 1, ey = (s >> 1) & 1;
      if (!((ex ? has_e : has_w) && (ey ? has_n : has_s))) continue;
      float t[ND];
      corner_taylor<2, P>(T, base + ex + ey * HX, NH, ex ? -1.0f : 1.0f, ey ? -1.0f : 1.0f, t);
      float b2 = 0.0f;
#pragma unroll
      for (int k = 1; k < ND; ++k) b2 = fmaf(T.sigma[k] * t[k], t[k], b2);
      const float wt = 1.0f / ipowf(a.eps + powq(sqrtf(b2), a.q), a.r);
      wsum += wt;
#pragma unroll
      for (int k = 0; k < ND; ++k) acc[k] = fmaf(wt, t[k], acc[k]);
    }
    const float inv = 1.0f / wsum;
#pragma unroll
    for (int k = 0; k < ND; ++k) st[k * NVT + vtx] = acc[k] * inv;
    if (a.tstar_out) {
      int I = i0 + va, J = j0 + vb;
      int vyn = a.pery ? ny : ny + 1;
      if ((va < TX || I == nx) && I < a.vx && (vb < TY || J == ny) && J < vyn) {
        size_t vi = (size_t)I + (size_t)a.vx * J;
#pragma unroll
        for (int k = 0; k < ND; ++k) a.tstar_out[vi * ND + k] = acc[k] * inv * T.tscale[k];
      }
    }
  }
  __syncthreads();

  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int gi = i0 + tx, gj = j0 + ty;
  if (gi >= nx || gj >= ny) return;
  const int hc = (ty + 1) * HX + tx + 1;
  const size_t cell = (size_t)gj * nx + gi;
  auto C = [&](int v, int m, int h) -> float { return sc[(v * ND + m) * NH + h]; };

  // ---- (c) sensor from the density -------------------------------------------------------
  float gam, n0;
  {
    float c[ND];
#pragma unroll
    for (int m = 0; m < ND; ++m) c[m] = C(0, m, hc);
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
    n0 = sqrtf(n0sq);
    const float om0 = (1.0f - NC * a.gamma_vertex) / ipowf(a.eps + powq(n0, a.q), a.r);
    float S[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) S[i] = om0 * w0[i];
    float osum = om0;
#pragma unroll
    for (int l = 0; l < NC; ++l) {
      const int vi = (tx + (l & 1)) + (ty + ((l >> 1) & 1)) * VXT;
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

  // ---- own traces at the face nodes (deviations from the cell mean), lambda_e ---------------
  bool bad = false;
  float Ubar[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) Ubar[v] = C(v, 0, hc);
  const EulerMean M = euler_mean(g, Ubar);
  float oR[NV][N], oL[NV][N], oT[NV][N], oB[NV][N];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    float trR[N], trL[N], trT[N], trB[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      float r = 0.0f, l = 0.0f, t = 0.0f, b = 0.0f;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const float cr = (i + N * j) ? C(v, i + N * j, hc) : 0.0f, ct = (j + N * i) ? C(v, j + N * i, hc) : 0.0f;
        r += cr;
        l += (i & 1) ? -cr : cr;
        t += ct;
        b += (i & 1) ? -ct : ct;
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
      oR[v][q] = r;
      oL[v][q] = l;
      oT[v][q] = t;
      oB[v][q] = b;
    }
  }
  float lam = 0.0f;
#pragma unroll
  for (int q = 0; q < N; ++q) {
    float U[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) U[v] = Ubar[v] + oR[v][q];
    lam = fmaxf(lam, euler_speed(g, U, bad));
#pragma unroll
    for (int v = 0; v < NV; ++v) U[v] = Ubar[v] + oL[v][q];
    lam = fmaxf(lam, euler_speed(g, U, bad));
#pragma unroll
    for (int v = 0; v < NV; ++v) U[v] = Ubar[v] + oT[v][q];
    lam = fmaxf(lam, euler_speed(g, U, bad));
#pragma unroll
    for (int v = 0; v < NV; ++v) U[v] = Ubar[v] + oB[v][q];
    lam = fmaxf(lam, euler_speed(g, U, bad));
  }
  // volume nodes: values, and the gradient data needed by stage (d)
  float gsq[NV][ND];  // |grad U_v|^2 at the volume nodes (physical)
#pragma unroll
  for (int qx = 0; qx < N; ++qx) {
    float tb[NV][N], td[NV][N];
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int my = 0; my < N; ++my) {
        float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
        for (int mx = 0; mx < N; ++mx) {
          s0 = fmaf(T.B[qx][mx], C(v, mx + N * my, hc), s0);
          s1 = fmaf(T.Bd[qx][mx], C(v, mx + N * my, hc), s1);
        }
        tb[v][my] = s0;
        td[v][my] = s1;
      }
#pragma unroll
    for (int qy = 0; qy < N; ++qy) {
      float U[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        float u = 0.0f, ux = 0.0f, uy = 0.0f;
#pragma unroll
        for (int my = 0; my < N; ++my) {
          u = fmaf(T.B[qy][my], tb[v][my], u);
          ux = fmaf(T.B[qy][my], td[v][my], ux);
          uy = fmaf(T.Bd[qy][my], tb[v][my], uy);
        }
        U[v] = u;
        ux *= a.two_dx;
        uy *= a.two_dy;
        gsq[v][qx + N * qy] = fmaf(ux, ux, uy * uy);
      }
      lam = fmaxf(lam, euler_speed(g, U, bad));
    }
  }
  const float nu = lam * a.nu_scale;
  if (a.gamma_out) a.gamma_out[cell] = gam;
  if (a.nu_out) a.nu_out[cell] = nu;
  if (a.lambda_out) a.lambda_out[cell] = lam;
  if (a.mode & kModeSensorOnly) {
    if (bad) atomicOr(a.status, kStatPositivity);
    return;
  }

  // ---- (d) SC weights: alpha~ from the density, f_q per variable -----------------------------
  bool troubled = a.sc && gam < a.c_gamma && n0 > 1e-30f;
  if (a.troubled_override) {
    int ov = a.troubled_override[cell];
    if (ov >= 0) troubled = ov && n0 > 1e-30f;
  }
  float Nq[ND];
  float afac[NV];  // alpha_{v,q} = Nq[q] * afac[v]; afac < 0 marks alpha = 1
#pragma unroll
  for (int v = 0; v < NV; ++v) afac[v] = -1.0f;
  if (troubled && gam < 1.0f) {
#pragma unroll
    for (int qx = 0; qx < N; ++qx) {
      float X[N][N];
#pragma unroll
      for (int kx = 0; kx < N; ++kx)
#pragma unroll
        for (int my = 0; my < N; ++my) {
          float acc = 0.0f;
#pragma unroll
          for (int mx = 0; mx < N; ++mx) acc = fmaf(T.Bk[kx][qx][mx], C(0, mx + N * my, hc), acc);
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
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      float s1 = 0.0f, s2 = 0.0f;
#pragma unroll
      for (int q = 0; q < ND; ++q) {
        const float W = T.w[q % N] * T.w[q / N];
        s1 = fmaf(W, gsq[v][q], s1);
        s2 = fmaf(W * Nq[q], gsq[v][q], s2);
      }
      if (s2 > 0.0f) afac[v] = s1 / s2;
    }
  }
  if (a.troubled_out) a.troubled_out[cell] = troubled ? 1 : 0;
  if (a.alpha_out) {
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int q = 0; q < ND; ++q) a.alpha_out[(cell * NV + v) * ND + q] = afac[v] >= 0.0f ? Nq[q] * afac[v] : 1.0f;
  }

  // ---- (e) residual ------------------------------------------------------------------------------
  float r[NV][ND];
  const float mu = (1.0f - gam) * nu;
  {
    const bool hasR = a.perx || gi + 1 < nx, hasL = a.perx || gi > 0;
    const bool hasT = a.pery || gj + 1 < ny, hasB = a.pery || gj > 0;
    // neighbour traces, projected to the face nodes one variable at a time
    float FR[NV][N], FL[NV][N], FT[NV][N], FB[NV][N];
    float vR[NV][N], vL[NV][N], vT[NV][N], vB[NV][N];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      float nR[N], nL[N], nT[N], nB[N];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        float r0 = 0.0f, l0 = 0.0f, t0 = 0.0f, b0 = 0.0f;
#pragma unroll
        for (int i = 0; i < N; ++i) {
          if (i + N * j) {
            const float cr = C(v, i + N * j, hc + 1), cl = C(v, i + N * j, hc - 1);
            r0 += (i & 1) ? -cr : cr;
            l0 += cl;
          }
          if (j + N * i) {
            const float ct = C(v, j + N * i, hc + HX), cb = C(v, j + N * i, hc - HX);
            t0 += (i & 1) ? -ct : ct;
            b0 += cb;
          }
        }
        nR[j] = r0;
        nL[j] = l0;
        nT[j] = t0;
        nB[j] = b0;
      }
#pragma unroll
      for (int q = 0; q < N; ++q) {
        float xr = 0.0f, xl = 0.0f, xt = 0.0f, xb = 0.0f;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          xr = fmaf(T.B[q][j], nR[j], xr);
          xl = fmaf(T.B[q][j], nL[j], xl);
          xt = fmaf(T.B[q][j], nT[j], xt);
          xb = fmaf(T.B[q][j], nB[j], xb);
        }
        vR[v][q] = hasR ? (C(v, 0, hc + 1) - Ubar[v]) + xr : oR[v][q];
        vL[v][q] = hasL ? (C(v, 0, hc - 1) - Ubar[v]) + xl : oL[v][q];
        vT[v][q] = hasT ? (C(v, 0, hc + HX) - Ubar[v]) + xt : oT[v][q];
        vB[v][q] = hasB ? (C(v, 0, hc - HX) - Ubar[v]) + xb : oB[v][q];
      }
    }
#pragma unroll
    for (int q = 0; q < N; ++q) {
      float UL[NV], UR[NV], F[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) { UL[v] = oR[v][q]; UR[v] = vR[v][q]; }
      hll_dev(g, M, UL, UR, 0, F, bad);
#pragma unroll
      for (int v = 0; v < NV; ++v) FR[v][q] = F[v];
#pragma unroll
      for (int v = 0; v < NV; ++v) { UL[v] = vL[v][q]; UR[v] = oL[v][q]; }
      hll_dev(g, M, UL, UR, 0, F, bad);
#pragma unroll
      for (int v = 0; v < NV; ++v) FL[v][q] = F[v];
#pragma unroll
      for (int v = 0; v < NV; ++v) { UL[v] = oT[v][q]; UR[v] = vT[v][q]; }
      hll_dev(g, M, UL, UR, 1, F, bad);
#pragma unroll
      for (int v = 0; v < NV; ++v) FT[v][q] = F[v];
#pragma unroll
      for (int v = 0; v < NV; ++v) { UL[v] = vB[v][q]; UR[v] = oB[v][q]; }
      hll_dev(g, M, UL, UR, 1, F, bad);
#pragma unroll
      for (int v = 0; v < NV; ++v) FB[v][q] = F[v];
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      float hR[N], hL[N], hT[N], hB[N];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
#pragma unroll
        for (int q = 0; q < N; ++q) {
          const float wb = T.w[q] * T.B[q][j];
          s0 = fmaf(wb, FR[v][q], s0);
          s1 = fmaf(wb, FL[v][q], s1);
          s2 = fmaf(wb, FT[v][q], s2);
          s3 = fmaf(wb, FB[v][q], s3);
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
          const float fxv = hR[my] - ((mx & 1) ? -hL[my] : hL[my]);
          const float fyv = hT[mx] - ((my & 1) ? -hB[mx] : hB[mx]);
          r[v][mx + N * my] = -(a.two_dx * fxv + a.two_dy * fyv);
        }
    }
  }
  // volume
#pragma unroll
  for (int qx = 0; qx < N; ++qx) {
    float tb[NV][N], td[NV][N];
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int my = 0; my < N; ++my) {
        float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
        for (int mx = 0; mx < N; ++mx) {
          const float cm = (mx + N * my) ? C(v, mx + N * my, hc) : 0.0f;  // deviation: no mean mode
          s0 = fmaf(T.B[qx][mx], cm, s0);
          s1 = fmaf(T.Bd[qx][mx], cm, s1);
        }
        tb[v][my] = s0;
        td[v][my] = s1;
      }
    float Gx[NV][N], Gy[NV][N];
#pragma unroll
    for (int qy = 0; qy < N; ++qy) {
      const int q = qx + N * qy;
      float dU[NV], Ux[NV], Uy[NV], Fx[NV], Fy[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        float u = 0.0f, ux = 0.0f, uy = 0.0f;
#pragma unroll
        for (int my = 0; my < N; ++my) {
          u = fmaf(T.B[qy][my], tb[v][my], u);
          ux = fmaf(T.B[qy][my], td[v][my], ux);
          uy = fmaf(T.Bd[qy][my], tb[v][my], uy);
        }
        dU[v] = u;
        Ux[v] = ux;
        Uy[v] = uy;
      }
      euler_dflux(g, M, dU, Fx, Fy);
      const float W = T.w[qx] * T.w[qy];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const float al = afac[v] >= 0.0f ? Nq[q] * afac[v] : 1.0f;
        Gx[v][qy] = W * (Fx[v] - mu * al * a.two_dx * Ux[v]);
        Gy[v][qy] = W * (Fy[v] - mu * al * a.two_dy * Uy[v]);
      }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      float hx[N], hy[N];
#pragma unroll
      for (int my = 0; my < N; ++my) {
        float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
        for (int qy = 0; qy < N; ++qy) {
          s0 = fmaf(T.B[qy][my], Gx[v][qy], s0);
          s1 = fmaf(T.Bd[qy][my], Gy[v][qy], s1);
        }
        hx[my] = s0;
        hy[my] = s1;
      }
#pragma unroll
      for (int my = 0; my < N; ++my)
#pragma unroll
        for (int mx = 0; mx < N; ++mx) {
          float val = r[v][mx + N * my];
          val = fmaf(a.two_dx * T.Bd[qx][mx], hx[my], val);
          val = fmaf(a.two_dy * T.B[qx][mx], hy[my], val);
          r[v][mx + N * my] = val;
        }
    }
  }
  // M^{-1}, output
  bool nonfinite = false;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    float* out = a.u_out + ((size_t)v * ncell + cell) * ND;
    const float* un = a.u_n + ((size_t)v * ncell + cell) * ND;
#pragma unroll
    for (int m = 0; m < ND; ++m) {
      const int mx = m % N, my = m / N;
      const float d = r[v][m] * (0.25f * (2 * mx + 1) * (2 * my + 1));
      nonfinite |= !isfinite(d);
      if (a.mode & kModeRK) {
        float val = fmaf(a.dt, d, C(v, m, hc));
        if (a.rk_a != 0.0f) val = fmaf(a.rk_b, val - un[m], un[m]);
        out[m] = val;
      } else {
        out[m] = d;
      }
    }
  }
  if (nonfinite) atomicOr(a.status, kStatNonfinite);
  if (bad) atomicOr(a.status, kStatPositivity);
}

template <int P, int TX, int TY>
cudaError_t launch_euler(const cvweno_mesh_s* m, const StageArgs& a, cudaStream_t s) {
  using Tb = DgTables<2, P>;
  constexpr size_t smem = sizeof(float) * ((size_t)NV * Tb::ND * (TX + 2) * (TY + 2) + (size_t)Tb::ND * (TX + 1) * (TY + 1));
  static_assert(smem <= 220 * 1024, "tile too large for shared memory");
  auto kern = dg_euler_stage<P, TX, TY>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (m->tables_bytes != sizeof(Tb)) return cudaErrorInvalidValue;
  dim3 grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY);
  kern<<<grid, TX * TY, smem, s>>>(a, *static_cast<const Tb*>(m->tables));
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_stage_euler(const cvweno_mesh_s* m, const StageArgs& a, cudaStream_t s) {
  if (m->dim != 2) return cudaErrorNotSupported;
  switch (m->p) {
    case 1: return launch_euler<1, 16, 8>(m, a, s);
    case 2: return launch_euler<2, 16, 8>(m, a, s);
    case 3: return launch_euler<3, 16, 8>(m, a, s);
    case 4: return launch_euler<4, 8, 8>(m, a, s);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace cvw
