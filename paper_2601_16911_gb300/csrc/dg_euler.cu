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
  float irho;       // 1 / rho of the mean
};

__device__ __forceinline__ EulerMean euler_mean(float g, const float* Ub) {
  EulerMean M;
#pragma unroll
  for (int v = 0; v < NV; ++v) M.U[v] = Ub[v];
  const float ir = 1.0f / Ub[0];
  M.irho = ir;
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
  const float ir = rcp_fast(rb * (rb + d[0]));
  const float dvx = diff_of_products(d[1], rb, M.U[1], d[0]) * ir;
  const float dvy = diff_of_products(d[2], rb, M.U[2], d[0]) * ir;
  // dE rhobar - (dmx mbarx + dmy mbary) / 2, compensated
  const float x1 = diff_of_products(d[3], rb, 0.5f * d[1], M.U[1]);
  const float p2 = 0.5f * d[2] * M.U[2];
  const float e2 = fmaf(0.5f * d[2], M.U[2], -p2);
  const float x = (x1 - p2) - e2;
  const float dEmK = x * M.irho - 0.5f * ((M.U[1] + d[1]) * dvx + (M.U[2] + d[2]) * dvy);
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

// |v| + c at a node of full state U, with the velocity along x (dir 0) or y (dir 1) and
// the sound speed c; flags non-positive density or pressure
__device__ __forceinline__ float euler_wave(float g, const float* U, int dir, float& vn, float& c, bool& bad) {
  const float rho = U[0], ir = rcp_fast(rho);
  const float vx = U[1] * ir, vy = U[2] * ir;
  const float p = (g - 1.0f) * (U[3] - 0.5f * (U[1] * vx + U[2] * vy));
  bad |= !(rho > 0.0f) || !(p > 0.0f);
  c = sqrt_fast(g * fmaxf(p, 0.0f) * fabsf(ir));
  vn = dir == 0 ? vx : vy;
  return sqrt_fast(vx * vx + vy * vy) + c;
}

// |v| + c at a node of full state U; flags non-positive density or pressure
__device__ __forceinline__ float euler_speed(float g, const float* U, bool& bad) {
  float vn, c;
  return euler_wave(g, U, 0, vn, c, bad);
}

// HLL flux minus F(Ubar) . n across a face with normal +x (dir 0) or +y (dir 1), from
// the left/lower state Ubar + dL to the right/upper state Ubar + dR (reading A14), with
// Davis wave speeds from the two node states' normal velocities vnl, vnr and sound speeds
// cl, cr (euler_wave).  The constant F(Ubar) drops out of every branch:
// (S_R F(Ubar) - S_L F(Ubar)) / (S_R - S_L) = F(Ubar).
__device__ __forceinline__ void hll_dev(float g, const EulerMean& M, const float* dL, const float* dR, float vnl,
                                        float cl, float vnr, float cr, int dir, float* F) {
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
    const float inv = rcp_fast(sr - sl);
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = (sr * fl[v] - sl * fr[v] + sl * sr * (dR[v] - dL[v])) * inv;
  }
}

// Shared-memory layout of the Euler stage tile (floats).
template <int P, int TX, int TY>
struct EulerLayout {
  static constexpr int N = P + 1, ND = N * N, NT = TX * TY;
  static constexpr int HX = TX + 2, HY = TY + 2, NH = HX * HY;
  static constexpr int NVT = (TX + 1) * (TY + 1);
  // the tile's faces: x-faces (TX + 1 per tile row), then y-faces (TX per row of TY + 1)
  static constexpr int NFX = (TX + 1) * TY, NFACE = NFX + TX * (TY + 1);
  // per face: the projected flux h[v][j] (NV x N), then the largest wave speed of the
  // left/lower and of the right/upper cell's trace over the face nodes
  static constexpr int FS = NV * N + 2;
  static constexpr int OFF_SC = 0;                     // [NV][ND][NH] tile + halo, mode-major
  static constexpr int OFF_ST = OFF_SC + NV * ND * NH;  // [ND][NVT] density vertex candidates (to the sensor)
  static constexpr int OFF_NQ = OFF_ST;                 // [ND][NT] pointwise density indicator (after the sensor)
  static constexpr int OFF_F = OFF_ST + ND * NVT;       // [FS][NFACE] face results, component-major
  // halo staging of two variables, cell-major (cells of whole 16-byte chunks only), over
  // the vertex and face regions, which are written after the load
  static constexpr int OFF_STG = OFF_ST;
  static constexpr int STG = ND % 4 == 0 ? 2 * NH * ND : 0;
  static constexpr int FLOATS = OFF_F + FS * NFACE > OFF_STG + STG ? OFF_F + FS * NFACE : OFF_STG + STG;
  static constexpr size_t BYTES = sizeof(float) * (size_t)FLOATS;
  static_assert(ND * NT <= ND * NVT, "the indicator must fit over the vertex candidates");
};

// After the vertex phase, each thread takes its cell's sensor and then a share of the
// tile's faces, each face once (rolled over faces and nodes): both cells' traces, HLL
// relative to the left/lower cell's mean, projection onto the tangential modes, and each
// side's largest wave speed over the face nodes.  Then one thread per cell, ordered so
// that nothing larger than one row of volume nodes is held at a time:
//   faces: the four projected fluxes into r (a left/lower face was projected relative to
//     the neighbour's mean, so the cell adds F(Ubar_nb) - F(Ubar) on the face's mean
//     mode), lambda_e over the face nodes;
//   volume pass A (rolled over node rows): flux deviation projected into r, lambda_e
//     over the volume nodes, and the two sums of stage (d) per variable;
//   volume pass B, only where the viscosity (1 - gamma_e) nu_e is non-zero: the
//     alpha-weighted viscous term.
// Minimum resident CTAs the register allocation must allow, from a sweep on the 512^2
// quadrants (stage time, ms: p = 2: 0.21 uncapped, 0.20 at 4 CTAs; p = 3: 0.45 uncapped,
// 0.41 at 3 CTAs; p = 4 (8x8 tiles): 0.97 uncapped, 1.15 at 6 CTAs).
template <int P, int TX, int TY>
constexpr int euler_min_ctas() {
  return P <= 2 ? 4 * (128 / (TX * TY)) : P == 3 ? 3 * (128 / (TX * TY)) : 1;
}

template <int P, int TX, int TY>
__global__ void __launch_bounds__(TX* TY, (euler_min_ctas<P, TX, TY>()))
    dg_euler_stage(const __grid_constant__ StageArgs a, const __grid_constant__ DgTables<2, P> T) {
  using Tb = DgTables<2, P>;
  using L = EulerLayout<P, TX, TY>;
  constexpr int N = P + 1, ND = Tb::ND, NS = Tb::NS, NC = 4;
  constexpr int NT = TX * TY;
  constexpr int HX = TX + 2, NH = HX * (TY + 2);
  constexpr int VXT = TX + 1, NVT = VXT * (TY + 1);
  extern __shared__ __align__(16) float smem[];
  float* sc = smem + L::OFF_SC;
  float* st = smem + L::OFF_ST;
  float* sNq = smem + L::OFF_NQ;
  const int nx = a.nx, ny = a.ny;
  const size_t ncell = (size_t)nx * ny;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const float g = a.gas_gamma;

  // ---- load tile + halo of all variables (asynchronous copies) ---------------------------
  // Cells of whole 16-byte chunks (Q1, Q3) in a 16-byte-aligned state: 16-byte copies,
  // two variables at a time, land cell-major in the staging area and are transposed to
  // the mode-major layout; otherwise 4-byte copies straight into sc.
  static_assert(L::OFF_STG % 4 == 0, "staging must be 16-byte aligned");
  if (ND % 4 == 0 && (reinterpret_cast<uintptr_t>(a.u_in) & 15) == 0) {
    constexpr int NQ4 = ND / 4, NCH = NH * NQ4;
    float* stg = smem + L::OFF_STG;
#pragma unroll 1
    for (int half = 0; half < NV / 2; ++half) {
      for (int f = threadIdx.x; f < 2 * NCH; f += NT) {
        const int vv = f / NCH, rem = f - vv * NCH, h = rem / NQ4, q = rem - h * NQ4;
        const int v = 2 * half + vv, r = h / HX, cc = h - r * HX;
        int gi = i0 - 1 + cc, gj = j0 - 1 + r;
        bool ok = true;
        if (gi < 0 || gi >= nx) {
          if (a.perx) gi = (gi + nx) % nx; else ok = false;
        }
        if (gj < 0 || gj >= ny) {
          if (a.pery) gj = (gj + ny) % ny; else ok = false;
        }
        ok = ok && CVW_SPAN(a.status, ((size_t)v * ncell + (size_t)gj * nx + gi) * ND + 4 * q, 4, a.lim_in);
        cp_async16z(stg + 4 * f, ok ? a.u_in + ((size_t)v * ncell + (size_t)gj * nx + gi) * ND + 4 * q : a.u_in,
                    ok ? 16 : 0);
      }
      cp_async_wait_all();
      __syncthreads();
      for (int f = threadIdx.x; f < 2 * NCH; f += NT) {
        const int vv = f / NCH, rem = f - vv * NCH, h = rem / NQ4, q = rem - h * NQ4;
        const float4 x = *reinterpret_cast<const float4*>(stg + 4 * f);
        float* d = sc + ((2 * half + vv) * ND + 4 * q) * NH + h;
        d[0] = x.x;
        d[NH] = x.y;
        d[2 * NH] = x.z;
        d[3 * NH] = x.w;
      }
      __syncthreads();
    }
  } else {
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
    ok = ok && CVW_SPAN(a.status, ((size_t)v * ncell + (size_t)gj * nx + gi) * ND + mm, 1, a.lim_in);
    cp_async4(sc + (v * ND + mm) * NH + r * HX + cc,
              ok ? a.u_in + ((size_t)v * ncell + (size_t)gj * nx + gi) * ND + mm : a.u_in, ok ? 4 : 0);
  }
  cp_async_wait_all();
  __syncthreads();
  }

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
      const float wt = rcp_fast(ipowf(a.eps + powq(sqrt_fast(b2), a.q), a.r));
      wsum += wt;
#pragma unroll
      for (int k = 0; k < ND; ++k) acc[k] = fmaf(wt, t[k], acc[k]);
    }
    const float inv = rcp_fast(wsum);
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

  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int gi = i0 + tx, gj = j0 + ty;
  const int hc = (ty + 1) * HX + tx + 1;
  const size_t cell = (size_t)gj * nx + gi;
  // (the checked build also checks the cell's index in the per-cell outputs and its span of
  // u_n and u_out in the last variable)
  const bool active = gi < nx && gj < ny && CVW_SPAN(a.status, cell, 1, a.lim_cell) &&
                      CVW_SPAN(a.status, ((size_t)(NV - 1) * ncell + cell) * ND, ND,
                               a.lim_in < a.lim_out ? a.lim_in : a.lim_out);
  auto C = [&](int v, int m, int h) -> float { return sc[(v * ND + m) * NH + h]; };
  const bool sensor_only = (a.mode & kModeSensorOnly) != 0;
  bool bad = false;

  // ---- the tile's faces, each once: traces, HLL, projection, each side's wave speed --------------
  // In the vertex phase's barrier interval (the face results do not overlap the vertex
  // candidates), from the block's last thread backwards: the vertex phase's extra round
  // falls on the first threads, the face phase's on the last.
  float* sF = smem + L::OFF_F;
#pragma unroll 1
  for (int f = NT - 1 - threadIdx.x; f < L::NFACE; f += NT) {
    int dirn, hl, hr;
    bool hasl, hasr, needed;
    if (f < L::NFX) {
      const int row = f / (TX + 1), col = f - row * (TX + 1);
      hl = (row + 1) * HX + col;
      hr = hl + 1;
      dirn = 0;
      const int gl = i0 - 1 + col;
      hasl = a.perx || gl >= 0;
      hasr = a.perx || gl + 1 < nx;
      needed = row < act_y && col <= act_x;  // a side of an active cell
    } else {
      const int h = f - L::NFX, row = h / TX, col = h - row * TX;
      hl = row * HX + col + 1;
      hr = hl + HX;
      dirn = 1;
      const int gl = j0 - 1 + row;
      hasl = a.pery || gl >= 0;
      hasr = a.pery || gl + 1 < ny;
      needed = col < act_x && row <= act_y;
    }
    if (!needed) continue;
    // tangential trace coefficients (non-mean modes): the left/lower cell meets the face
    // with its upper side (+1), the right/upper cell with its lower side ((-1)^i along the
    // normal); a missing side (transmissive boundary) is the other side's ghost
    float tl[NV][N], tr[NV][N], UL[NV], UR[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
#pragma unroll
      for (int j = 0; j < N; ++j) {
        float sl = 0.0f, sr = 0.0f;
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const int m = dirn == 0 ? i + N * j : j + N * i;
          if (m == 0) continue;
          const float cl = C(v, m, hl), cr = C(v, m, hr);
          sl += cl;
          sr += (i & 1) ? -cr : cr;
        }
        tl[v][j] = sl;
        tr[v][j] = sr;
      }
      UL[v] = C(v, 0, hl);
      UR[v] = C(v, 0, hr);
    }
    if (!hasl) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        UL[v] = UR[v];
#pragma unroll
        for (int j = 0; j < N; ++j) tl[v][j] = tr[v][j];
      }
    }
    if (!hasr) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        UR[v] = UL[v];
#pragma unroll
        for (int j = 0; j < N; ++j) tr[v][j] = tl[v][j];
      }
    }
    const EulerMean ML = euler_mean(g, UL);
    float dm[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) dm[v] = UR[v] - UL[v];
    float h[NV][N];
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int j = 0; j < N; ++j) h[v][j] = 0.0f;
    float laml = 0.0f, lamr = 0.0f;
#pragma unroll 1
    for (int q = 0; q < N; ++q) {
      float dL[NV], dR[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        float sl = 0.0f, sr = 0.0f;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const float bq = T.B[q][j];
          sl = fmaf(bq, tl[v][j], sl);
          sr = fmaf(bq, tr[v][j], sr);
        }
        dL[v] = sl;
        dR[v] = sr;
      }
      float vnl, cl, vnr, cr;
      {
        float U[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) U[v] = UL[v] + dL[v];
        laml = fmaxf(laml, euler_wave(g, U, dirn, vnl, cl, bad));
#pragma unroll
        for (int v = 0; v < NV; ++v) U[v] = UR[v] + dR[v];
        lamr = fmaxf(lamr, euler_wave(g, U, dirn, vnr, cr, bad));
      }
      if (sensor_only) continue;
#pragma unroll
      for (int v = 0; v < NV; ++v) dR[v] = dm[v] + dR[v];
      float F[NV];
      hll_dev(g, ML, dL, dR, vnl, cl, vnr, cr, dirn, F);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const float wf = T.w[q] * F[v];
#pragma unroll
        for (int j = 0; j < N; ++j) h[v][j] = fmaf(wf, T.B[q][j], h[v][j]);
      }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int j = 0; j < N; ++j) sF[(v * N + j) * L::NFACE + f] = h[v][j];
    sF[NV * N * L::NFACE + f] = laml;
    sF[(NV * N + 1) * L::NFACE + f] = lamr;
  }
  __syncthreads();

  // ---- (c) sensor from the density -------------------------------------------------------
  float gam = 1.0f, n0 = 0.0f;
  if (active) {
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
    n0 = sqrt_fast(n0sq);
    const float om0 = (1.0f - NC * a.gamma_vertex) * rcp_fast(ipowf(a.eps + powq(n0, a.q), a.r));
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
      const float om = a.gamma_vertex * rcp_fast(ipowf(a.eps + powq(sqrt_fast(b2), a.q), a.r));
      osum += om;
#pragma unroll
      for (int i = 0; i < NS; ++i) S[i] = fmaf(om, wl[i], S[i]);
    }
    const float inv = rcp_fast(osum);
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
      gam = 1.0f - powq(fminf(1.0f, sqrt_fast(d2) * rcp_fast(n0)), a.q);
  }

  // the indicator sNq, written below, lies over the vertex candidates that the sensor reads
  __syncthreads();
  if (!active) {
    if (bad) atomicOr(a.status, kStatPositivity);
    return;
  }

  // ---- faces into the residual: right, left, top, bottom; lambda_e over the face nodes ---------
  float Ubar[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) Ubar[v] = C(v, 0, hc);
  const EulerMean M = euler_mean(g, Ubar);
  float r[NV][ND];
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int m = 0; m < ND; ++m) r[v][m] = 0.0f;
  float lam = 0.0f;
#pragma unroll 1
  for (int k = 0; k < 4; ++k) {
    const int dirn = k >> 1;
    const bool upper = (k & 1) == 0;  // this cell is the face's left/lower cell
    const int f = dirn == 0 ? ty * (TX + 1) + tx + (upper ? 1 : 0) : L::NFX + (ty + (upper ? 1 : 0)) * TX + tx;
    lam = fmaxf(lam, sF[(NV * N + (upper ? 0 : 1)) * L::NFACE + f]);
    if (sensor_only) continue;
    float h[NV][N];
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int j = 0; j < N; ++j) h[v][j] = sF[(v * N + j) * L::NFACE + f];
    const bool nb = dirn == 0 ? (a.perx || gi > 0) : (a.pery || gj > 0);
    if (!upper && nb) {
      // projected relative to the neighbour's mean: F - F(Ubar) = (F - F(Ubar_nb)) + D with
      // D = F(Ubar_nb) - F(Ubar) constant along the face, whose projection is 2 D on mode 0
      float d[NV], dFx[NV], dFy[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) d[v] = C(v, 0, hc - (dirn == 0 ? 1 : HX)) - Ubar[v];
      euler_dflux(g, M, d, dFx, dFy);
#pragma unroll
      for (int v = 0; v < NV; ++v) h[v][0] = fmaf(2.0f, dirn == 0 ? dFx[v] : dFy[v], h[v][0]);
    }
    // r[mx,my] -= 2/dx (hR[my] - (-1)^mx hL[my]) + 2/dy (hT[mx] - (-1)^my hB[mx])
    const float s2d = dirn == 0 ? a.two_dx : a.two_dy;
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int my = 0; my < N; ++my)
#pragma unroll
        for (int mx = 0; mx < N; ++mx) {
          const int nrm = dirn == 0 ? mx : my;
          const float hv = dirn == 0 ? h[v][my] : h[v][mx];
          r[v][mx + N * my] = upper ? fmaf(-s2d, hv, r[v][mx + N * my])
                                    : fmaf(s2d, (nrm & 1) ? -hv : hv, r[v][mx + N * my]);
        }
  }

  // ---- troubled cells: the density's pointwise indicator Nq at the volume nodes -------------
  bool troubled = a.sc && gam < a.c_gamma && n0 > 1e-30f;
  if (!sensor_only && a.troubled_override) {
    const int ov = a.troubled_override[cell];
    if (ov >= 0) troubled = ov && n0 > 1e-30f;
  }
  const bool need_sc = !sensor_only && troubled && gam < 1.0f;
  if (need_sc) {
#pragma unroll 1
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
#pragma unroll 1
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
        sNq[(qx + N * qy) * NT + threadIdx.x] = sqrtf(s2);
      }
    }
  }

  // ---- volume pass A: flux deviation into r, lambda_e, the sums of stage (d) ----------------
  float s1[NV], s2[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) s1[v] = s2[v] = 0.0f;
#pragma unroll 1
  for (int qx = 0; qx < N; ++qx) {
    float tb[NV][N], td[NV][N];
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int my = 0; my < N; ++my) {
        float s0 = 0.0f, sd = 0.0f;
#pragma unroll
        for (int mx = 0; mx < N; ++mx) {
          const float cm = (mx + N * my) ? C(v, mx + N * my, hc) : 0.0f;  // deviation: no mean mode
          s0 = fmaf(T.B[qx][mx], cm, s0);
          sd = fmaf(T.Bd[qx][mx], cm, sd);
        }
        tb[v][my] = s0;
        td[v][my] = sd;
      }
    float hx[NV][N], hy[NV][N];
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int my = 0; my < N; ++my) hx[v][my] = hy[v][my] = 0.0f;
#pragma unroll 1
    for (int qy = 0; qy < N; ++qy) {
      const int q = qx + N * qy;
      const float W = T.w[qx] * T.w[qy];
      float dU[NV];
      const float nq = need_sc ? sNq[q * NT + threadIdx.x] : 0.0f;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        float u = 0.0f, ux = 0.0f, uy = 0.0f;
#pragma unroll
        for (int my = 0; my < N; ++my) {
          const float bq = T.B[qy][my];
          u = fmaf(bq, tb[v][my], u);
          ux = fmaf(bq, td[v][my], ux);
          uy = fmaf(T.Bd[qy][my], tb[v][my], uy);
        }
        dU[v] = u;
        if (need_sc) {
          ux *= a.two_dx;
          uy *= a.two_dy;
          const float gsq = fmaf(ux, ux, uy * uy);
          s1[v] = fmaf(W, gsq, s1[v]);
          s2[v] = fmaf(W * nq, gsq, s2[v]);
        }
      }
      {
        float U[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) U[v] = Ubar[v] + dU[v];
        lam = fmaxf(lam, euler_speed(g, U, bad));
      }
      if (sensor_only) continue;
      float Fx[NV], Fy[NV];
      euler_dflux(g, M, dU, Fx, Fy);
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int my = 0; my < N; ++my) {
          hx[v][my] = fmaf(W * Fx[v], T.B[qy][my], hx[v][my]);
          hy[v][my] = fmaf(W * Fy[v], T.Bd[qy][my], hy[v][my]);
        }
    }
    if (sensor_only) continue;
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int my = 0; my < N; ++my)
#pragma unroll
        for (int mx = 0; mx < N; ++mx) {
          float val = r[v][mx + N * my];
          val = fmaf(a.two_dx * T.Bd[qx][mx], hx[v][my], val);
          val = fmaf(a.two_dy * T.B[qx][mx], hy[v][my], val);
          r[v][mx + N * my] = val;
        }
  }
  const float nu = lam * a.nu_scale;
  if (a.gamma_out) a.gamma_out[cell] = gam;
  if (a.nu_out) a.nu_out[cell] = nu;
  if (a.lambda_out) a.lambda_out[cell] = lam;
  if (sensor_only) {
    if (bad) atomicOr(a.status, kStatPositivity);
    return;
  }

  // ---- (d) SC weights: alpha_{v,q} = Nq[q] afac[v] (afac < 0: alpha = 1) ------------------------
  float afac[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) afac[v] = (need_sc && s2[v] > 0.0f) ? s1[v] / s2[v] : -1.0f;
  if (a.troubled_out) a.troubled_out[cell] = troubled ? 1 : 0;
  if (a.alpha_out) {
#pragma unroll 1
    for (int q = 0; q < ND; ++q) {
      const float nq = need_sc ? sNq[q * NT + threadIdx.x] : 0.0f;
#pragma unroll
      for (int v = 0; v < NV; ++v) a.alpha_out[(cell * NV + v) * ND + q] = afac[v] >= 0.0f ? nq * afac[v] : 1.0f;
    }
  }

  // ---- volume pass B: the viscous term, where (1 - gamma_e) nu_e > 0 -----------------------------
  // With the linear weights (alpha = 1 for every variable) the term is -mu times the
  // stiffness form of the Legendre basis, which the Gauss rule integrates exactly and which
  // separates: the x part of mode (mx, my) is (2/dx)^2 (2 / (2 my + 1)) sum_k S[mx][k]
  // c[k, my], with S[m][k] = int P_m' P_k' = min(m,k) (min(m,k) + 1) where m + k is even
  // (0 otherwise), and likewise in y.  Alpha-weighted cells take the quadrature.
  const float mu = (1.0f - gam) * nu;
  bool weighted = false;
#pragma unroll
  for (int v = 0; v < NV; ++v) weighted |= afac[v] >= 0.0f;
  if (mu > 0.0f && !weighted) {
    const float kx = -mu * a.two_dx * a.two_dx, ky = -mu * a.two_dy * a.two_dy;
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
      for (int my = 0; my < N; ++my)
#pragma unroll
        for (int mx = 0; mx < N; ++mx) {
          if (mx + my == 0) continue;
          float sx = 0.0f, sy = 0.0f;
#pragma unroll
          for (int k = 1; k < N; ++k) {
            if ((k + mx) % 2 == 0 && mx > 0) {
              const int mn = mx < k ? mx : k;
              sx = fmaf((float)(mn * (mn + 1)), C(v, k + N * my, hc), sx);
            }
            if ((k + my) % 2 == 0 && my > 0) {
              const int mn = my < k ? my : k;
              sy = fmaf((float)(mn * (mn + 1)), C(v, mx + N * k, hc), sy);
            }
          }
          const float val = fmaf(kx * (2.0f / (2 * my + 1)), sx, r[v][mx + N * my]);
          r[v][mx + N * my] = fmaf(ky * (2.0f / (2 * mx + 1)), sy, val);
        }
  } else if (mu > 0.0f) {
#pragma unroll 1
    for (int qx = 0; qx < N; ++qx) {
      float tb[NV][N], td[NV][N];
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int my = 0; my < N; ++my) {
          float s0 = 0.0f, sd = 0.0f;
#pragma unroll
          for (int mx = 0; mx < N; ++mx) {
            const float cm = (mx + N * my) ? C(v, mx + N * my, hc) : 0.0f;
            s0 = fmaf(T.B[qx][mx], cm, s0);
            sd = fmaf(T.Bd[qx][mx], cm, sd);
          }
          tb[v][my] = s0;
          td[v][my] = sd;
        }
      float hx[NV][N], hy[NV][N];
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int my = 0; my < N; ++my) hx[v][my] = hy[v][my] = 0.0f;
#pragma unroll 1
      for (int qy = 0; qy < N; ++qy) {
        const int q = qx + N * qy;
        const float W = T.w[qx] * T.w[qy];
        const float nq = need_sc ? sNq[q * NT + threadIdx.x] : 0.0f;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          float ux = 0.0f, uy = 0.0f;
#pragma unroll
          for (int my = 0; my < N; ++my) {
            ux = fmaf(T.B[qy][my], td[v][my], ux);
            uy = fmaf(T.Bd[qy][my], tb[v][my], uy);
          }
          const float al = afac[v] >= 0.0f ? nq * afac[v] : 1.0f;
          const float gx = -W * mu * al * a.two_dx * ux, gy = -W * mu * al * a.two_dy * uy;
#pragma unroll
          for (int my = 0; my < N; ++my) {
            hx[v][my] = fmaf(gx, T.B[qy][my], hx[v][my]);
            hy[v][my] = fmaf(gy, T.Bd[qy][my], hy[v][my]);
          }
        }
      }
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int my = 0; my < N; ++my)
#pragma unroll
          for (int mx = 0; mx < N; ++mx) {
            float val = r[v][mx + N * my];
            val = fmaf(a.two_dx * T.Bd[qx][mx], hx[v][my], val);
            val = fmaf(a.two_dy * T.B[qx][mx], hy[v][my], val);
            r[v][mx + N * my] = val;
          }
    }
  }

  // ---- M^{-1}, output ---------------------------------------------------------------------------
  // Per variable, the cell's u_n is read in full before any of its outputs is written: only
  // this thread reads or writes the cell's span, so u_n may alias u_out, and the reads of a
  // variable go out together instead of one round trip per mode.  16-byte loads and stores
  // where the cell is whole 16-byte chunks and both states are 16-byte aligned.
  bool nonfinite = false;
  const bool rk = (a.mode & kModeRK) != 0, with_un = rk && a.rk_a != 0.0f;
  const bool v16 = ND % 4 == 0 && ((reinterpret_cast<uintptr_t>(a.u_out) | reinterpret_cast<uintptr_t>(a.u_n)) & 15) == 0;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    float* out = a.u_out + ((size_t)v * ncell + cell) * ND;
    const float* un = a.u_n + ((size_t)v * ncell + cell) * ND;
    float o[ND];
    if (with_un) {
      if (v16) {
#pragma unroll
        for (int q = 0; q < ND / 4; ++q) {
          const float4 x = reinterpret_cast<const float4*>(un)[q];
          o[4 * q] = x.x;
          o[4 * q + 1] = x.y;
          o[4 * q + 2] = x.z;
          o[4 * q + 3] = x.w;
        }
      } else {
#pragma unroll
        for (int m = 0; m < ND; ++m) o[m] = un[m];
      }
    }
#pragma unroll
    for (int m = 0; m < ND; ++m) {
      const int mx = m % N, my = m / N;
      const float d = r[v][m] * (0.25f * (2 * mx + 1) * (2 * my + 1));
      nonfinite |= !isfinite(d);
      if (rk) {
        float val = fmaf(a.dt, d, C(v, m, hc));
        if (with_un) val = fmaf(a.rk_b, val - o[m], o[m]);
        o[m] = val;
      } else {
        o[m] = d;
      }
    }
    if (v16) {
#pragma unroll
      for (int q = 0; q < ND / 4; ++q)
        reinterpret_cast<float4*>(out)[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
    } else {
#pragma unroll
      for (int m = 0; m < ND; ++m) out[m] = o[m];
    }
  }
  if (nonfinite) atomicOr(a.status, kStatNonfinite);
  if (bad) atomicOr(a.status, kStatPositivity);
}

template <int P, int TX, int TY>
cudaError_t launch_euler(const cvweno_mesh_s* m, const StageArgs& a, cudaStream_t s) {
  using Tb = DgTables<2, P>;
  constexpr size_t smem = EulerLayout<P, TX, TY>::BYTES;
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


// ---- positivity limiter (readings P1-P4; Zhang and Shu's scaling limiter) --------------------
// One thread per cell, cell-local (no neighbours, so it may run in place).  The cell's
// coefficients of all four variables are staged in shared memory (mode-major per
// thread); every volume and face Gauss node is evaluated from them, the density's
// non-mean modes are scaled to keep rho >= eps_e, then all non-mean modes to keep
// p >= eps_e, the root of p(U_bar + t dU) = eps_e found by 40 bisection steps.
template <int P>
struct PosThreads {
  static constexpr int value = P >= 4 ? 64 : 128;  // the staged coefficients stay under 48 KB
};

template <int P>
__global__ void __launch_bounds__(PosThreads<P>::value)
    euler_positivity_kernel(const __grid_constant__ StageArgs a, const __grid_constant__ DgTables<2, P> T,
                            float* __restrict__ theta_out) {
  constexpr int N = P + 1, ND = N * N, NTH = PosThreads<P>::value;
  __shared__ float sc[NV * ND][NTH];
  const int64_t ncell = (int64_t)a.nx * a.ny;
  const int64_t cell = (int64_t)blockIdx.x * NTH + threadIdx.x;
  if (cell >= ncell) return;
  if (!CVW_SPAN(a.status, cell, 1, a.lim_cell) ||
      !CVW_SPAN(a.status, ((NV - 1) * ncell + cell) * ND, ND, a.lim_in < a.lim_out ? a.lim_in : a.lim_out))
    return;
  const float g = a.gas_gamma;
#pragma unroll 1
  for (int k = 0; k < NV * ND; ++k) {
    const int v = k / ND, m = k - v * ND;
    sc[k][threadIdx.x] = a.u_in[((int64_t)v * ncell + cell) * ND + m];
  }
  float Ub[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) Ub[v] = sc[v * ND][threadIdx.x];
  const float pb = (g - 1.0f) * (Ub[3] - 0.5f * (Ub[1] * Ub[1] + Ub[2] * Ub[2]) / Ub[0]);
  float th1 = 1.0f, th2 = 1.0f;
  const bool admissible = Ub[0] > 0.0f && pb > 0.0f;
  if (admissible) {
    const float eps = 1e-3f * fminf(Ub[0], pb);
    // node q: volume (q < N^2: qx + N qy), then faces x = +1, x = -1, y = +1, y = -1
    auto value = [&](int v, int q) -> float {
      float s = 0.0f;
#pragma unroll 1
      for (int my = 0; my < N; ++my) {
        float row = 0.0f;
#pragma unroll
        for (int mx = 0; mx < N; ++mx) {
          float bx;
          if (q < ND) bx = T.B[q % N][mx];
          else if (q < ND + 2 * N) bx = (q < ND + N || !(mx & 1)) ? 1.0f : -1.0f;
          else bx = T.B[(q - ND) % N][mx];
          row = fmaf(bx, sc[v * ND + mx + N * my][threadIdx.x], row);
        }
        float by;
        if (q < ND) by = T.B[q / N][my];
        else if (q < ND + 2 * N) by = T.B[(q - ND) % N][my];
        else by = (q < ND + 3 * N || !(my & 1)) ? 1.0f : -1.0f;
        s = fmaf(by, row, s);
      }
      return s;
    };
    constexpr int NPT = ND + 4 * N;
    float rmin = Ub[0];
#pragma unroll 1
    for (int q = 0; q < NPT; ++q) rmin = fminf(rmin, value(0, q));
    if (rmin < eps) th1 = fminf(1.0f, (Ub[0] - eps) / (Ub[0] - rmin));
    auto pres = [&](const float* U) {
      return (g - 1.0f) * (U[3] - 0.5f * (U[1] * U[1] + U[2] * U[2]) / U[0]);
    };
#pragma unroll 1
    for (int q = 0; q < NPT; ++q) {
      float Uq[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) Uq[v] = value(v, q);
      Uq[0] = fmaf(th1, Uq[0] - Ub[0], Ub[0]);
      if (!(pres(Uq) < eps)) continue;
      float lo = 0.0f, hi = 1.0f;  // p(lo) >= eps > p(hi)
#pragma unroll 1
      for (int it = 0; it < 40; ++it) {
        const float t = 0.5f * (lo + hi);
        float Ut[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) Ut[v] = fmaf(t, Uq[v] - Ub[v], Ub[v]);
        if (pres(Ut) >= eps) lo = t; else hi = t;
      }
      th2 = fminf(th2, lo);
    }
  } else {
    atomicOr(a.status, kStatPositivity);
  }
#pragma unroll 1
  for (int k = 0; k < NV * ND; ++k) {
    const int v = k / ND, m = k - v * ND;
    const float f = m == 0 ? 1.0f : (v == 0 ? th1 : 1.0f) * th2;
    a.u_out[((int64_t)v * ncell + cell) * ND + m] = sc[k][threadIdx.x] * f;
  }
  if (theta_out) theta_out[cell] = th1 * th2;
}

template <int P>
cudaError_t launch_positivity_p(const cvweno_mesh_s* m, const StageArgs& a, float* theta, cudaStream_t s) {
  using Tb = DgTables<2, P>;
  if (m->tables_bytes != sizeof(Tb)) return cudaErrorInvalidValue;
  const int64_t ncell = (int64_t)a.nx * a.ny;
  constexpr int nth = PosThreads<P>::value;
  euler_positivity_kernel<P><<<(unsigned)((ncell + nth - 1) / nth), nth, 0, s>>>(a, *static_cast<const Tb*>(m->tables),
                                                                                  theta);
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

cudaError_t launch_positivity(const cvweno_mesh_s* m, const StageArgs& a, float* theta, cudaStream_t s) {
  if (m->dim != 2 || m->desc.system != CVWENO_EULER || m->kind != CVWENO_DG) return cudaErrorNotSupported;
  switch (m->p) {
    case 1: return launch_positivity_p<1>(m, a, theta, s);
    case 2: return launch_positivity_p<2>(m, a, theta, s);
    case 3: return launch_positivity_p<3>(m, a, theta, s);
    case 4: return launch_positivity_p<4>(m, a, theta, s);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace cvw
