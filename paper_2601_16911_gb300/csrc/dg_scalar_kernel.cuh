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
// Code-size discipline: the loops over vertex slots, corners, face nodes and volume
// nodes are rolled and read their tabulations (staged in shared memory) with uniform,
// broadcast loads, so the kernel body stays within the instruction cache; only the
// short loops over modes are unrolled into registers.  All arithmetic is FP32.
#pragma once

#include <utility>

#include "cvweno_internal.cuh"
#include "mlp_mma.cuh"
#include "tc_tf32.cuh"

namespace cvw {

__device__ __forceinline__ float ipowf(float x, int r) {
  if (r == 2) return x * x;  // the paper's r
  float y = x;
  for (int i = 1; i < r; ++i) y *= x;
  return y;
}

// The general power is out of line: it is cold at the paper's q = 1, and inlined at every
// call site it crowds the instruction cache of the stage kernels.
static __device__ __noinline__ float powf_cold(float x, float q) { return powf(x, q); }
__device__ __forceinline__ float powq(float x, float q) { return q == 1.0f ? x : powf_cold(x, q); }

// Reciprocal and square root in PTX's approximate forms (relative error about 2^-22, no
// range check and no slow path), for the nonlinear weights and norms of stages (b)-(c)
// and the node-wise flux paths, which need FP32 precision, not correct rounding.
__device__ __forceinline__ float rcp_fast(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ float sqrt_fast(float x) {
  float y;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

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
  __device__ __forceinline__ void flux_mean(float& fx, float& fy) const { fx = fy = 0.5f * ubar * ubar; }
  // |f'(u)| (Euclidean) for nu_e, and |f'(u) . n| for an axis-aligned face
  __device__ __forceinline__ float speed(float u) const { return DIM == 2 ? 1.41421356237f * fabsf(u) : fabsf(u); }
  __device__ __forceinline__ float nspeed(float u, int) const { return fabsf(u); }
};

// sin d and cos d - 1 for |d| <= 1 from their Maclaurin series, Horner in d^2, to the
// d^11 and d^12 terms: the first omitted terms are below 2e-10 at |d| = 1, far under one
// FP32 ulp, and cos d - 1 comes without cancellation.
__device__ __forceinline__ void sin_cosm1_small(float d, float& s, float& cm1) {
  const float z = d * d;
  float ps = fmaf(z, -1.0f / 39916800.0f, 1.0f / 362880.0f);
  ps = fmaf(z, ps, -1.0f / 5040.0f);
  ps = fmaf(z, ps, 1.0f / 120.0f);
  ps = fmaf(z, ps, -1.0f / 6.0f);
  s = fmaf(d * z, ps, d);
  float pc = fmaf(z, 1.0f / 479001600.0f, -1.0f / 3628800.0f);
  pc = fmaf(z, pc, 1.0f / 40320.0f);
  pc = fmaf(z, pc, -1.0f / 720.0f);
  pc = fmaf(z, pc, 1.0f / 24.0f);
  pc = fmaf(z, pc, -0.5f);
  cm1 = z * pc;
}

// sin d and cos d - 1 for the deviations beyond |d| = 1 (a few multiples of pi inside a
// KPP cell): Cody and Waite's reduction d = k pi/2 + r, |r| <= pi/4, with pi/2 split into
// an FP32 head and tail and the FMA products exact, then the series above for r and the
// quadrant k mod 4.  cos d - 1 is taken from cos r - 1 where cos d = cos r (no
// cancellation); in the other quadrants cos d is at most cos(pi/4) and c - 1 does not
// cancel.  Accurate to a few FP32 ulps while k pi/2's tail stays below half an ulp of r,
// i.e. for |d| up to about 1e3 (a KPP state lies within [pi/4, 7 pi/2] by the maximum
// principle); a non-finite d gives non-finite results, which the stage flags.
__device__ __forceinline__ void sin_cosm1_reduced(float d, float& s, float& cm1) {
  const float k = rintf(d * 0.636619772f);      // nearest multiple of pi/2
  float r = fmaf(-k, 1.57079637f, d);            // pi/2 rounded to FP32 ...
  r = fmaf(-k, -4.37113883e-8f, r);              // ... and the rest of pi/2
  float sr, cr1;
  sin_cosm1_small(r, sr, cr1);
  switch ((int)k & 3) {
    case 0: s = sr; cm1 = cr1; break;
    case 1: s = cr1 + 1.0f; cm1 = -sr - 1.0f; break;
    case 2: s = -sr; cm1 = -cr1 - 2.0f; break;
    default: s = -(cr1 + 1.0f); cm1 = sr - 1.0f; break;
  }
}

template <int DIM>
struct ScalarLaw<CVWENO_KPP, DIM> {
  float sb, cb;  // sin(ubar), cos(ubar)
  __device__ __forceinline__ ScalarLaw(const StageArgs&, float ub) {
    float cm1;
    sin_cosm1_reduced(ub, sb, cm1);
    cb = 1.0f + cm1;
  }
  // sin(ub + d) - sin(ub) = sin(ub)(cos d - 1) + cos(ub) sin d, and likewise for cos.
  // Deviations inside a cell are mostly small: the series above; otherwise the reduced
  // series (sin_cosm1_reduced).
  __device__ __forceinline__ void flux_dev(float d, float& fx, float& fy) const {
    float s, cm1;
    if (fabsf(d) <= 1.0f) {
      sin_cosm1_small(d, s, cm1);
    } else {
      sin_cosm1_reduced(d, s, cm1);
    }
    fx = fmaf(sb, cm1, cb * s);
    fy = fmaf(cb, cm1, -sb * s);
  }
  __device__ __forceinline__ float flux_dev_dir(float d, int dir) const {
    float fx, fy;
    flux_dev(d, fx, fy);
    return dir == 0 ? fx : fy;
  }
  __device__ __forceinline__ void flux_mean(float& fx, float& fy) const {
    fx = sb;
    fy = cb;
  }
  __device__ __forceinline__ float speed(float) const { return 1.0f; }
  __device__ __forceinline__ float nspeed(float u, int dir) const {
    return dir == 0 ? fabsf(cosf(u)) : fabsf(sinf(u));
  }
};

template <int DIM>
struct ScalarLaw<CVWENO_LINADV, DIM> {
  float vx, vy, ubar;
  __device__ __forceinline__ ScalarLaw(const StageArgs& a, float ub) : vx(a.adv_vx), vy(a.adv_vy), ubar(ub) {}
  __device__ __forceinline__ void flux_mean(float& fx, float& fy) const {
    fx = vx * ubar;
    fy = vy * ubar;
  }
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

// Reference Taylor data t[k] = d^k u (sx, sy) at corner (sx, sy) in {-1, 1}^2 of one
// cell whose coefficients sit at c[m * stride]:
//   t[kx + N ky] = sx^kx sy^ky sum_my E[ky][my] sy^my sum_mx E[kx][mx] sx^mx c[mx, my]
// using P_m^(k)(-1) = (-1)^(m+k) P_m^(k)(1).
template <int DIM, int P>
__device__ __forceinline__ void corner_taylor(const DgTables<DIM, P>& T, const float* c, int stride, float sx, float sy,
                                              float* t) {
  constexpr int N = P + 1;
  float px[N], py[N];
  px[0] = py[0] = 1.0f;
#pragma unroll
  for (int m = 1; m < N; ++m) {
    px[m] = px[m - 1] * sx;
    py[m] = py[m - 1] * sy;
  }
  if constexpr (DIM == 1) {
    float cl[N];
#pragma unroll
    for (int m = 0; m < N; ++m) cl[m] = c[m * stride] * px[m];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      float acc = 0.0f;
#pragma unroll
      for (int m = 0; m < N; ++m) acc = fmaf(T.E[k][m], cl[m], acc);
      t[k] = acc * px[k];
    }
  } else {
    float cl[N * N];
#pragma unroll
    for (int my = 0; my < N; ++my)
#pragma unroll
      for (int mx = 0; mx < N; ++mx) cl[mx + N * my] = c[(mx + N * my) * stride] * (px[mx] * py[my]);
    float tmp[N][N];  // [kx][my]
#pragma unroll
    for (int kx = 0; kx < N; ++kx)
#pragma unroll
      for (int my = 0; my < N; ++my) {
        float acc = 0.0f;
#pragma unroll
        for (int mx = 0; mx < N; ++mx) acc = fmaf(T.E[kx][mx], cl[mx + N * my], acc);
        tmp[kx][my] = acc;
      }
#pragma unroll
    for (int ky = 0; ky < N; ++ky)
#pragma unroll
      for (int kx = 0; kx < N; ++kx) {
        float acc = 0.0f;
#pragma unroll
        for (int my = 0; my < N; ++my) acc = fmaf(T.E[ky][my], tmp[kx][my], acc);
        t[kx + N * ky] = acc * (px[kx] * py[ky]);
      }
  }
}

// Shared-memory layout of the tile: halo coefficients, vertex candidates, the corner
// matrices (rows padded to a multiple of 4 floats for 16-byte broadcast loads), the
// 1D tabulations read with run-time node indices, and per-thread alpha~ storage.
// TC: the tensor-core form of the sensor (2D, p = 3, 8 x 16 tiles).  The vertex
// candidates are kept only as the split TF32 MMA operand [part][K chunk][vertex][4]
// (16-byte rows, vertex-major within a chunk), which for every corner l is a canonical
// operand over the tile's cells as it stands: the cells of a tile row (8, one core-matrix
// group) meet 8 consecutive vertices, and the next tile row starts VXT vertices further
// on (the descriptor's 8-row-group stride).  The image is staged from B on, with its
// tensor-core section (the split corner matrices); the alpha~ storage reuses the operand
// once the MMAs have completed.
template <int DIM, int P, int TX, int TY, bool TC = false>
struct TileLayout {
  using Tb = DgTables<DIM, P>;
  static constexpr int N = P + 1, ND = Tb::ND, NS = Tb::NS, NC = Tb::NC;
  using Img = TabImage<DIM, P>;
  static constexpr int NSP = Img::NSP;
  static constexpr int NT = TX * TY;
  static constexpr int HX = TX + 2, HY = DIM == 2 ? TY + 2 : 1, NH = HX * HY;
  static constexpr int VXT = TX + 1, VYT = DIM == 2 ? TY + 1 : 1, NVT = VXT * VYT;
  static_assert(!TC || (Img::HAS_TC && TX == 8 && NT == 128), "tensor-core form: 2D p = 3, 8 x 16 tiles");
  static constexpr int TCK = Img::TCK, TCCH = TCK / 4;            // K of the corner products, its 16-byte chunks
  static constexpr int TSA_PART = TCCH * NVT * 4;                 // floats of one part (hi or lo) of the operand
  static constexpr int OFF_SC = 0;                                // [ND][NH]
  static constexpr int OFF_ST = OFF_SC + ND * NH;                 // [ND][NVT]
  static constexpr int OFF_TSA = (OFF_SC + ND * NH + 3) / 4 * 4;  // TC: [2][TCCH][NVT][4]
  // the staged TabImage (16-byte aligned): A [NC][NS][NSP], B[q][m], Bd[q][m],
  // Bk[k][q][m], w[q] (TC: from B on, then the tensor-core section); image float f sits
  // at OFF_A + f
  static constexpr int IMG0 = TC ? Img::B : 0;
  static constexpr int IMG1 = TC ? Img::FLOATS_ALL : Img::FLOATS;
  static constexpr int OFF_A = (TC ? OFF_TSA + 2 * TSA_PART : (OFF_ST + ND * NVT + 3) / 4 * 4) - IMG0;
  static constexpr int OFF_B = OFF_A + Img::B;
  static constexpr int OFF_BD = OFF_A + Img::BD;
  static constexpr int OFF_BK = OFF_A + Img::BK;
  static constexpr int OFF_W = OFF_A + Img::W;
  static constexpr int OFF_ATC = OFF_A + Img::TC;                 // TC: [2][NC][TCCH][TCK][4]
  static constexpr int OFF_NQ = TC ? OFF_TSA : OFF_A + Img::FLOATS;  // [ND][NT] pointwise indicators
  static constexpr int OFF_UN = TC ? OFF_A + IMG1 : OFF_NQ + ND * NT;  // u_n of the tile's cells, [ND][NT] or [NT][ND]
  // the tile's loads are staged over the indicator and u_n regions (TC: over the operand)
  static constexpr int STAGING = TC ? 2 * TSA_PART : 2 * ND * NT;
  static_assert(!TC || ND * NT <= 2 * TSA_PART, "alpha~ storage must fit the operand region");
  // face fluxes of the tile, projected on the tangential modes: x-faces ((TX+1) per tile
  // row), then y-faces (TX per row, TY+1 rows)
  // (degrees 2 and 3, from measurements: at p = 1 the face work per cell is too small to
  // pay for the face phase's own law evaluations and its uneven rounds before the
  // barrier; at p = 4 the batch kernel, at its register cap, lost time; the surrogate
  // instantiation at p = 2, held to 96 registers, keeps the cell-wise faces)
  static constexpr bool SHARED_FACES = P == 2 || P == 3;
  static constexpr int NFP = DIM == 2 ? N : 1;
  static constexpr int NFX = (TX + 1) * TY, NFY = DIM == 2 ? TX * (TY + 1) : 0, NFACE = NFX + NFY;
  static constexpr int OFF_F = OFF_UN + ND * NT;                  // [NFACE][NFP]
  static constexpr int FLOATS = OFF_F + (SHARED_FACES ? NFACE * NFP : 0);
  static constexpr size_t BYTES = sizeof(float) * (size_t)FLOATS;
  // with the surrogate sensor: packed weights, then one 32 x 16 bf16 input block per warp
  static constexpr int OFF_MLP = (FLOATS + 3) / 4 * 4;
  static constexpr int OFF_XS = OFF_MLP + (int)(sizeof(MlpPacked) / sizeof(float));
  static constexpr size_t BYTES_MLP = sizeof(float) * (size_t)OFF_XS + (size_t)(NT / 32) * 32 * 16 * 2;
};

// 4-byte asynchronous global -> shared copy (zero-filled when src_bytes == 0), so that a
// thread keeps all of its tile loads in flight at once instead of waiting on each.
__device__ __forceinline__ void cp_async4(float* dst, const float* src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Copies the packed surrogate weights into shared memory (uint4 copies; NB threads).
template <int DIM, int P, int TX, int TY, int NB = TX * TY>
__device__ __forceinline__ void stage_mlp_to_smem(const void* mlp, float* smem) {
  using L = TileLayout<DIM, P, TX, TY>;
  const uint4* src = static_cast<const uint4*>(mlp);
  uint4* dst = reinterpret_cast<uint4*>(smem + L::OFF_MLP);
  for (int i = threadIdx.x; i < (int)(sizeof(MlpPacked) / 16); i += NB) dst[i] = __ldg(src + i);
}

// Surrogate inputs of one cell (2D): per corner l, the vertex candidate's cell mean minus
// the cell mean, and its h-scaled gradient at the vertex, over ||u^e||_e + eps, clamped to
// [-8, 8].  st holds reference-coordinate Taylor data; the cell mean of the Taylor
// monomial (xi - s)^k / k! over [-1, 1] is (-s)^k 2^k / (k+1)!.
template <int P, int TX, int TY>
__device__ __forceinline__ void cell_features(const StageArgs& a, const float* st, float c0, float n0, int tx,
                                              int ty, float (&f)[kMlpIn]) {
  using L = TileLayout<2, P, TX, TY>;
  constexpr int N = L::N, VXT = L::VXT, NVT = L::NVT;
  float mom[N];
  {
    float v = 1.0f, fact = 1.0f;
#pragma unroll
    for (int k = 0; k < N; ++k) {  // 2^k / (k+1)!
      fact *= (float)(k + 1);
      mom[k] = v / fact;
      v *= 2.0f;
    }
  }
  const float inv_s = 1.0f / (n0 + a.eps);
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    const int vi = (tx + (l & 1)) + (ty + (l >> 1)) * VXT;
    const float sx = (l & 1) ? -1.0f : 1.0f, sy = (l & 2) ? -1.0f : 1.0f;
    float mean = 0.0f;
#pragma unroll
    for (int ky = 0; ky < N; ++ky) {
      float row = 0.0f;
      float px = 1.0f;
#pragma unroll
      for (int kx = 0; kx < N; ++kx) {
        row = fmaf(st[(kx + N * ky) * NVT + vi] * px, mom[kx], row);
        px *= sx;
      }
      mean = fmaf(row, mom[ky] * ((ky & 1) ? sy : 1.0f), mean);
    }
    const float gx = a.h_e * a.two_dx * st[1 * NVT + vi], gy = a.h_e * a.two_dy * st[N * NVT + vi];
    f[3 * l + 0] = fminf(8.0f, fmaxf(-8.0f, (mean - c0) * inv_s));
    f[3 * l + 1] = fminf(8.0f, fmaxf(-8.0f, gx * inv_s));
    f[3 * l + 2] = fminf(8.0f, fmaxf(-8.0f, gy * inv_s));
  }
}

// Reading S7: with the surrogate, a cell whose semi-norm is below this fraction of
// (|mean| + 1) holds rounding-level variation only; it takes gamma_e = 1 directly.
constexpr float kNearFlat = 1e-5f;

template <int DIM, int P>
__device__ __forceinline__ float cell_norm0(const DgTables<DIM, P>& T, const float* c) {
  constexpr int NS = DgTables<DIM, P>::NS;
  float n2 = 0.0f;
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    float acc = 0.0f;
#pragma unroll
    for (int j = i; j < NS; ++j) acc = fmaf(T.R[i][j], c[j + 1], acc);
    n2 = fmaf(acc, acc, n2);
  }
  return sqrtf(n2);
}

// Programmatic dependent launch.  A stage kernel launched with programmatic stream
// serialisation may start while the previous kernel on its stream finishes: before
// pdl_wait() it touches only data that no kernel of the current step writes (the
// tabulation image, shared memory); pdl_wait() returns once the previous kernel has
// completed and its writes are visible.  pdl_launch_dependents() lets the next kernel
// start once every CTA of this one has passed it.  Both are no-ops without the launch
// attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// Host: launches kern with programmatic stream serialisation, so that it may start while
// the previous kernel on stream s finishes (the kernel must call pdl_wait() before it
// touches anything that kernel writes).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// 16-byte asynchronous global -> shared copy (both addresses 16-byte aligned); the
// zero-filling form copies src_bytes (0 or 16) and fills the rest with zeros.
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cp_async16z(float* dst, const float* src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes));
}

// Starts the copy of R rows of W consecutive columns of a row-major global array (nrow
// rows of ncol columns, each column E floats) into shared memory: row r, column c lands at
// dst[r * RS + ph[r] + c * E + e].  Global row r0 + r and column c0 + c wrap (periodic) or,
// outside the array, read as zeros.  The row's in-range columns are one run in global
// memory; ph[r] is its offset within a 16-byte chunk, so the run's whole chunks are copied
// 16 bytes at a time (src 16-byte aligned required) and only its head and tail (under 4
// floats each, 6 at most when the run has no whole chunk) and the wrapped or absent
// columns float by float.  One warp per row (rows of many chunks).  Requires
// RS >= W * E + 3; the copies land with the thread's next cp.async wait, the zeros and
// ph[] with the next barrier.
template <int E, int W, int R, int RS, int NT>
__device__ __forceinline__ void stage_rows16(float* dst, int* ph, const float* src, int ncol, int nrow, int c0,
                                             int r0, bool perc, bool perr, int* status, int64_t lim) {
  static_assert(RS >= W * E + 3 && RS % 4 == 0, "staging row too short");
  constexpr int NW = NT / 32;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int c_lo = max(0, -c0), c_hi = min(W - 1, ncol - 1 - c0);  // in-range columns
  const int cr = max(c_hi + 1, c_lo), nout = (c_lo + W - cr) * E;  // columns [0, c_lo), [cr, W)
#pragma unroll 1
  for (int r = warp; r < R; r += NW) {
    int gr = r0 + r;
    bool row_ok = true;
    if (gr < 0 || gr >= nrow) {
      if (perr) gr = ((gr % nrow) + nrow) % nrow; else row_ok = false;
    }
    float* d = dst + r * RS;
    if (!row_ok) {
      for (int e = lane; e < W * E; e += 32) d[e] = 0.0f;
      if (lane == 0) ph[r] = 0;
      continue;
    }
    const int64_t gbase = ((int64_t)gr * ncol + c0) * E;  // global float of column 0
    const int p = (int)(gbase & 3);
    if (lane == 0) ph[r] = p;
    d += p;
    const int64_t dofs = (int64_t)r * RS + p - gbase;  // staging float of global float x: x + dofs
    // body: the whole 16-byte chunks of the in-range run [g0, g1)
    const int64_t g0 = gbase + (int64_t)c_lo * E, g1 = c_hi < c_lo ? g0 : gbase + (int64_t)(c_hi + 1) * E;
    const int64_t b0 = (g0 + 3) & ~(int64_t)3, b1 = g1 & ~(int64_t)3;
    const bool body = b0 < b1;
    if (body)
      for (int64_t x = b0 + 4 * lane; x < b1; x += 128)
        if (CVW_SPAN(status, x, 4, lim) && CVW_SPAN(status, x + dofs, 4, R * RS)) cp_async16(d + (x - gbase), src + x);
    // head and tail of the run (or the whole run when it has no whole chunk)
    const int nh = body ? (int)(b0 - g0) : (int)(g1 - g0), nt = body ? (int)(g1 - b1) : 0;
    if (lane < nh) {
      if (CVW_SPAN(status, g0 + lane, 1, lim) && CVW_SPAN(status, g0 + lane + dofs, 1, R * RS))
        cp_async4(d + (g0 + lane - gbase), src + g0 + lane, 4);
    } else if (lane < nh + nt) {
      if (CVW_SPAN(status, b1 + lane - nh, 1, lim) && CVW_SPAN(status, b1 + lane - nh + dofs, 1, R * RS))
        cp_async4(d + (b1 + lane - nh - gbase), src + b1 + lane - nh, 4);
    }
    for (int j = lane; j < nout; j += 32) {
      const int cj = j / E, e = j - cj * E;
      const int c = cj < c_lo ? cj : cr + (cj - c_lo);
      if (perc) {
        const int gc = ((c0 + c) % ncol + ncol) % ncol;
        if (CVW_SPAN(status, ((int64_t)gr * ncol + gc) * E + e, 1, lim) &&
            CVW_SPAN(status, (int64_t)r * RS + p + c * E + e, 1, R * RS))
          cp_async4(d + c * E + e, src + ((int64_t)gr * ncol + gc) * E + e, 4);
      } else {
        d[c * E + e] = 0.0f;
      }
    }
  }
}

// Starts the copy of the tabulation image img (device, TabImage<DIM, P>) into shared
// memory; it lands with the tile's first cp.async wait.  NB: threads of the block.
template <int DIM, int P, int TX, int TY, int NB = TX * TY, bool TC = false>
__device__ __forceinline__ void stage_tables_to_smem(const float* img, float* smem) {
  using L = TileLayout<DIM, P, TX, TY, TC>;
  for (int f = L::IMG0 / 4 + threadIdx.x; f < L::IMG1 / 4; f += NB) cp_async16(smem + L::OFF_A + 4 * f, img + 4 * f);
}

// Writes TabImage<DIM, P> of T to img (one block; run once per mesh, off the stage path).
template <int DIM, int P>
__global__ void tab_image_kernel(const __grid_constant__ DgTables<DIM, P> T, float* __restrict__ img) {
  using I = TabImage<DIM, P>;
  constexpr int N = I::N, NS = I::NS, NSP = I::NSP;
  for (int f = threadIdx.x; f < I::FLOATS_ALL; f += blockDim.x) {
    float v = 0.0f;
    if (f >= I::TC) {  // split corner matrix: [part][l][K chunk j][row i][e], K index 4 j + e
      constexpr int TCK = I::TCK, NC = I::NC;
      const int g = f - I::TC, part = g / (NC * TCK * TCK), r = g - part * (NC * TCK * TCK);
      const int l = r / (TCK * TCK), r2 = r - l * (TCK * TCK), j = r2 / (4 * TCK), r3 = r2 - j * (4 * TCK);
      const int i = r3 / 4, k = 4 * j + (r3 & 3);
      const float x = (i < NS && k < NS) ? (&T.A[0][0][0])[(l * NS + i) * NS + k] : 0.0f;
      const float hi = tc::tf32_rna(x);
      v = part == 0 ? hi : tc::tf32_rna(x - hi);
    } else if (f < I::B) {
      const int l = f / (NS * NSP), rem = f - l * (NS * NSP), i = rem / NSP, j = rem - i * NSP;
      v = j < NS ? T.A[l][i][j] : 0.0f;
    } else if (f < I::BD) {
      v = (&T.B[0][0])[f - I::B];
    } else if (f < I::BK) {
      v = (&T.Bd[0][0])[f - I::BD];
    } else if (f < I::W) {
      v = (&T.Bk[0][0][0])[f - I::BK];
    } else if (f < I::W + N) {
      v = T.w[f - I::W];
    }
    img[f] = v;
  }
}

// Stages (a)+(b) for the tile's vertices, from the halo coefficients sc (mode-major):
// vertex candidates t* into st, and (optionally) the physical vertex data to tstar_out.
// NB threads of the block share the vertices.
template <int DIM, int P, int TX, int TY, int NB = TX * TY, bool TC = false>
__device__ __forceinline__ void tile_vertex_phase(const StageArgs& a, const DgTables<DIM, P>& T, const float* sc,
                                                  float* st, int i0, int j0, int nx, int ny) {
  using L = TileLayout<DIM, P, TX, TY, TC>;
  constexpr int ND = L::ND, NC = L::NC, HX = L::HX, NH = L::NH, VXT = L::VXT, NVT = L::NVT;
  const int act_x = min(TX, nx - i0), act_y = DIM == 2 ? min(TY, ny - j0) : 1;
  for (int v = threadIdx.x; v < NVT; v += NB) {
    int va = v % VXT, vb = DIM == 2 ? v / VXT : 0;
    if (va > act_x || (DIM == 2 && vb > act_y)) continue;
    float acc[ND];
#pragma unroll
    for (int k = 0; k < ND; ++k) acc[k] = 0.0f;
    float wsum = 0.0f;
    const int gi_w = i0 - 1 + va, gj_s = j0 - 1 + vb;
    const bool has_w = a.perx || gi_w >= 0, has_e = a.perx || gi_w + 1 < nx;
    const bool has_s = DIM == 1 || a.pery || gj_s >= 0, has_n = DIM == 1 || a.pery || gj_s + 1 < ny;
    const float* base = sc + (DIM == 2 ? vb * HX : 0) + va;
    // slots SW, SE, NW, NE: the cell right of / above the vertex touches it with its
    // left / lower corner (sign -1), the cell left of / below with its right / upper one
#pragma unroll (DIM == 1 || P <= 2 ? NC : 1)
    for (int s = 0; s < NC; ++s) {
      const int ex = s & 1, ey = (s >> 1) & 1;
      if (!((ex ? has_e : has_w) && (ey ? has_n : has_s))) continue;
      float t[ND];
      corner_taylor<DIM, P>(T, base + ex + (DIM == 2 ? ey * HX : 0), NH, ex ? -1.0f : 1.0f, ey ? -1.0f : 1.0f, t);
      float b2 = 0.0f;
#pragma unroll
      for (int k = 1; k < ND; ++k) b2 = fmaf(T.sigma[k] * t[k], t[k], b2);
      const float wt = rcp_fast(ipowf(a.eps + powq(sqrt_fast(b2), a.q), a.r));
      wsum += wt;
#pragma unroll
      for (int k = 0; k < ND; ++k) acc[k] = fmaf(wt, t[k], acc[k]);
    }
    const float inv = rcp_fast(wsum);
    if constexpr (TC) {
      // t*_1 .. t*_NS, zero-padded to TCK, split into TF32 hi and lo: row v of the operand
#pragma unroll
      for (int j = 0; j < L::TCCH; ++j) {
        float hi[4], lo[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int k = 4 * j + e + 1;
          tc::split_tf32(k < ND ? acc[k < ND ? k : 0] * inv : 0.0f, hi[e], lo[e]);
        }
        *reinterpret_cast<float4*>(st + (j * NVT + v) * 4) = make_float4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<float4*>(st + L::TSA_PART + (j * NVT + v) * 4) = make_float4(lo[0], lo[1], lo[2], lo[3]);
      }
    } else {
#pragma unroll
      for (int k = 0; k < ND; ++k) st[k * NVT + v] = acc[k] * inv;
    }
    if (a.tstar_out) {
      int I = i0 + va, J = j0 + vb;
      bool own_x = (va < TX || I == nx) && I < a.vx;
      int vyn = DIM == 2 ? (a.pery ? ny : ny + 1) : 1;
      bool own_y = DIM == 1 || ((vb < TY || J == ny) && J < vyn);
      if (own_x && own_y) {
        size_t vi = (size_t)I + (size_t)a.vx * J;
        if (CVW_SPAN(a.status, vi * ND, ND, (int64_t)a.vx * vyn * ND))
#pragma unroll
          for (int k = 0; k < ND; ++k) a.tstar_out[vi * ND + k] = acc[k] * inv * T.tscale[k];
      }
    }
  }
}

// Stage (c) for one cell with Legendre coefficients c: the cell-vertex reconstruction
// and the sensor gamma_e (eq. gamma); n0 returns ||u^e||_e.
template <int DIM, int P, int TX, int TY>
__device__ __forceinline__ float cell_sensor(const StageArgs& a, const DgTables<DIM, P>& T, const float* st,
                                             const float* sA, const float* c, int tx, int ty, float& n0,
                                             float* wstar) {
  using L = TileLayout<DIM, P, TX, TY>;
  constexpr int NS = L::NS, NC = L::NC, NSP = L::NSP, VXT = L::VXT, NVT = L::NVT;
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
#pragma unroll (DIM == 1 || P <= 2 ? NC : 1)
  for (int l = 0; l < NC; ++l) {
    const int vi = (tx + (l & 1)) + (DIM == 2 ? (ty + ((l >> 1) & 1)) * VXT : 0);
    float tl[NSP];
#pragma unroll
    for (int k = 0; k < NSP; ++k) tl[k] = k < NS ? st[(k + 1) * NVT + vi] : 0.0f;
    const float4* Al = reinterpret_cast<const float4*>(sA + l * NS * NSP);
    float wl[NS];
    float b2 = 0.0f;
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      float acc = 0.0f;
#pragma unroll
      for (int j4 = 0; j4 < NSP / 4; ++j4) {
        const float4 q4 = Al[i * (NSP / 4) + j4];
        acc = fmaf(q4.x, tl[4 * j4 + 0], acc);
        acc = fmaf(q4.y, tl[4 * j4 + 1], acc);
        acc = fmaf(q4.z, tl[4 * j4 + 2], acc);
        acc = fmaf(q4.w, tl[4 * j4 + 3], acc);
      }
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
    wstar[i] = S[i] * inv;  // semi-norm coordinates of u^{e,*} (dead unless the limiter reads it)
    d2 = fmaf(df, df, d2);
  }
  // the limiter, the surrogate's inputs and its fallback always use the computed sensor
  const bool forced = !(a.mode & (kModeLimit | kModeFeatures));
  if (forced && a.sensor_mode == CVWENO_SENSOR_SMOOTH) return 1.0f;
  if (forced && a.sensor_mode == CVWENO_SENSOR_TROUBLED) return 0.0f;
  if (n0 <= 1e-30f) return 1.0f;
  return 1.0f - powq(fminf(1.0f, sqrt_fast(d2) * rcp_fast(n0)), a.q);
}

// Tensor memory and completion barrier of the tensor-core form of the sensor (one
// allocation per CTA, made before the tile and freed inside it).
struct TcCtx {
  const uint32_t* slot;  // shared: TMEM base address (lane 0, first of kTcCols columns)
  uint32_t mbar;         // shared-memory address of the MMA completion mbarrier
  uint32_t* done;        // shared: warps that have read their corner products
};
constexpr uint32_t kTcCols = 64;          // 4 corners x 16 FP32 columns
constexpr uint32_t kTcPolls = 1u << 22;   // bounded wait for the corner products

// Issued by one thread once the tile's vertex candidates (the split operand) are in
// shared memory: w_l = A[l] t*_l for the four corners l of all 128 cells, into TMEM
// columns 16 l .. 16 l + 15 of the cell's lane, as A_hi B_hi + A_hi B_lo + A_lo B_hi.
template <int P, int TX, int TY>
__device__ __forceinline__ void issue_corner_products(const float* smem, const TcCtx& tcx) {
  using L = TileLayout<2, P, TX, TY, true>;
  constexpr int TCK = L::TCK, NC = L::NC;
  constexpr uint32_t ALBO = L::NVT * 16, ASBO = L::VXT * 16, APART = L::TSA_PART * 4;
  constexpr uint32_t BLBO = TCK * 16, BSBO = 8 * 16, BCORNER = TCK * TCK * 4, BPART = NC * BCORNER;
  const uint32_t id = tc::idesc_tf32(128, TCK);
  const uint32_t tsa = tc::smem_u32(smem + L::OFF_TSA), atc = tc::smem_u32(smem + L::OFF_ATC);
  tc::fence_after();
  const uint32_t tmem = *tcx.slot;
#pragma unroll
  for (int l = 0; l < NC; ++l) {
    const uint32_t a0 = tsa + (((l >> 1) & 1) * L::VXT + (l & 1)) * 16, b0 = atc + l * BCORNER;
    const uint32_t d = tmem + 16 * l;
#pragma unroll
    for (int s = 0; s < TCK / 8; ++s) {
      const uint64_t ah = tc::smem_desc(a0 + 2 * s * ALBO, ALBO, ASBO);
      const uint64_t al = tc::smem_desc(a0 + APART + 2 * s * ALBO, ALBO, ASBO);
      const uint64_t bh = tc::smem_desc(b0 + 2 * s * BLBO, BLBO, BSBO);
      const uint64_t bl = tc::smem_desc(b0 + BPART + 2 * s * BLBO, BLBO, BSBO);
      tc::mma_tf32(d, ah, bh, id, s > 0);
      tc::mma_tf32(d, ah, bl, id, 1u);
      tc::mma_tf32(d, al, bh, id, 1u);
    }
  }
  tc::commit(tcx.mbar);
}

// Stage (c) as cell_sensor, with the corner products A[l] t*_l read from tensor memory
// (issue_corner_products).  Every thread of the CTA calls it (the TMEM loads are
// warp-collective), cells outside the mesh included; the last warp to have read its
// products frees the TMEM.  overlap() runs between the cell's own part and the wait for
// the tensor cores: work of the cell that does not depend on the sensor.
template <int DIM, int P, int TX, int TY, class Overlap>
__device__ __forceinline__ float cell_sensor_tc(const StageArgs& a, const DgTables<DIM, P>& T, const TcCtx& tcx,
                                                const float* c, float& n0, float* wstar, Overlap&& overlap) {
  using L = TileLayout<DIM, P, TX, TY, true>;
  constexpr int NS = L::NS, NC = L::NC;
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
  overlap();
  if (!tc::mbar_wait(tcx.mbar, 0, kTcPolls)) atomicOr(a.status, kStatTimeout);
  tc::fence_after();
  const uint32_t tmem = *tcx.slot;
  const uint32_t trow = tmem + ((threadIdx.x & ~31u) << 16);
#pragma unroll 1
  for (int l = 0; l < NC; ++l) {
    float wl[16];
    tc::tmem_ld16(trow + 16 * l, wl);
    float b2 = 0.0f;
#pragma unroll
    for (int i = 0; i < NS; ++i) b2 = fmaf(wl[i], wl[i], b2);
    const float om = a.gamma_vertex * rcp_fast(ipowf(a.eps + powq(sqrt_fast(b2), a.q), a.r));
    osum += om;
#pragma unroll
    for (int i = 0; i < NS; ++i) S[i] = fmaf(om, wl[i], S[i]);
  }
  // this warp is done with the TMEM; the last of the CTA's warps frees it
  tc::fence_before();
  __syncwarp();
  uint32_t arrived = 0;
  if ((threadIdx.x & 31) == 0) {
    __threadfence_block();
    arrived = atomicAdd(tcx.done, 1u);
  }
  arrived = __shfl_sync(0xffffffffu, arrived, 0);
  if (arrived == TX * TY / 32 - 1) {
    __threadfence_block();
    tc::fence_after();
    tc::tmem_dealloc(tmem, kTcCols);
  }
  const float inv = rcp_fast(osum);
  float d2 = 0.0f;
#pragma unroll
  for (int i = 0; i < NS; ++i) {
    float df = w0[i] - S[i] * inv;
    wstar[i] = S[i] * inv;
    d2 = fmaf(df, df, d2);
  }
  const bool forced = !(a.mode & (kModeLimit | kModeFeatures));
  if (forced && a.sensor_mode == CVWENO_SENSOR_SMOOTH) return 1.0f;
  if (forced && a.sensor_mode == CVWENO_SENSOR_TROUBLED) return 0.0f;
  if (n0 <= 1e-30f) return 1.0f;
  return 1.0f - powq(fminf(1.0f, sqrt_fast(d2) * rcp_fast(n0)), a.q);
}

// Stage (e), faces: every face of the tile once (the cell-wise loop saw each interior face
// from both sides).  The LLF flux at the face's Gauss nodes minus f(ubar_l) . n, ubar_l the
// mean of the left/lower cell (of the right/upper one where the left/lower cell is absent
// at a transmissive boundary, whose ghost is the present cell's trace), projected onto the
// tangential Legendre modes: sF[face][j] = sum_q w_q P_j(xi_q) F_q.  The right/upper cell
// adds the difference of the two means' fluxes (mode 0 only).
template <int DIM, int P, int SYS, int TX, int TY, int NB = TX * TY>
__device__ __forceinline__ void tile_face_phase(const StageArgs& a, const float* sc, const float* sB, const float* sW,
                                                float* sF, int i0, int j0, int nx, int ny) {
  using L = TileLayout<DIM, P, TX, TY>;
  using Law = ScalarLaw<SYS, DIM>;
  constexpr int N = L::N, NH = L::NH, HX = L::HX, NFX = L::NFX, NFACE = L::NFACE, NFP = L::NFP;
  // faces from the block's last thread backwards: the vertex phase's extra round falls on
  // the first warp, the face phase's on the last
#pragma unroll 1
  for (int f = NB - 1 - threadIdx.x; f < NFACE; f += NB) {
    int dirn, hl, hr;
    bool hasl, hasr;
    if (f < NFX) {
      const int row = f / (TX + 1), col = f - row * (TX + 1);
      hl = (DIM == 2 ? (row + 1) * HX : 0) + col;
      hr = hl + 1;
      dirn = 0;
      const int gl = i0 - 1 + col;
      hasl = a.perx || gl >= 0;
      hasr = a.perx || gl + 1 < nx;
    } else {
      const int g = f - NFX, row = g / TX, col = g - row * TX;
      hl = row * HX + col + 1;
      hr = hl + HX;
      dirn = 1;
      const int gl = j0 - 1 + row;
      hasl = a.pery || gl >= 0;
      hasr = a.pery || gl + 1 < ny;
    }
    // traces along the face, relative to each cell's own mean: the left/lower cell meets
    // the face with its right/upper side (+1), the right/upper cell with its left/lower
    // side ((-1)^i along the normal)
    float tl[NFP], tr[NFP];
#pragma unroll
    for (int j = 0; j < NFP; ++j) {
      float sl = 0.0f, sr = 0.0f;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int m = DIM == 1 ? i : (dirn == 0 ? i + N * j : j + N * i);
        if (m == 0) continue;
        const float vr = sc[m * NH + hr];
        sl += sc[m * NH + hl];
        sr += (i & 1) ? -vr : vr;
      }
      tl[j] = sl;
      tr[j] = sr;
    }
    float ul = sc[hl], ur = sc[hr];
    if (!hasl) {
#pragma unroll
      for (int j = 0; j < NFP; ++j) tl[j] = tr[j];
      ul = ur;
    }
    if (!hasr) {
#pragma unroll
      for (int j = 0; j < NFP; ++j) tr[j] = tl[j];
      ur = ul;
    }
    const Law law(a, ul);
    const float dm = ur - ul;
    float h[NFP];
#pragma unroll
    for (int j = 0; j < NFP; ++j) h[j] = 0.0f;
#pragma unroll 1
    for (int q = 0; q < NFP; ++q) {
      float vl = tl[0], vr = tr[0];
      if constexpr (DIM == 2) {
        vl = vr = 0.0f;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const float bq = sB[q * N + j];
          vl = fmaf(bq, tl[j], vl);
          vr = fmaf(bq, tr[j], vr);
        }
      }
      const float F = llf_dev(law, a, ul, vl, dm + vr, dirn);
      if constexpr (DIM == 2) {
        const float wq = sW[q] * F;
#pragma unroll
        for (int j = 0; j < N; ++j) h[j] = fmaf(wq, sB[q * N + j], h[j]);
      } else {
        h[0] = F;
      }
    }
#pragma unroll
    for (int j = 0; j < NFP; ++j) sF[f * NFP + j] = h[j];
  }
}

// Stage (e), the faces' part of a cell's residual from the tile's face phase (sF): a lower
// face (left/bottom) was projected relative to the neighbour's mean, so this cell adds
// f(ubar_nb) - f(ubar) (mode 0: the integral of P_j over the face is 2 delta_j0) where that
// neighbour is present.  r is accumulated.
template <int DIM, int P, int SYS, int TX, int TY, bool TC>
__device__ __forceinline__ void shared_face_residual(const StageArgs& a, const ScalarLaw<SYS, DIM>& law,
                                                     const float* smem, const float* sc, float ubar, int tx, int ty,
                                                     int gi, int gj, int hc, float* r) {
  using L = TileLayout<DIM, P, TX, TY, TC>;
  constexpr int N = L::N, HX = L::HX;
  const float* sF = smem + L::OFF_F;
  if constexpr (DIM == 1) {
    const bool hasL = a.perx || gi > 0;
    const float FR = sF[tx + 1];
    const float FL = sF[tx] + (hasL ? law.flux_dev_dir(sc[hc - 1] - ubar, 0) : 0.0f);
#pragma unroll
    for (int m = 0; m < N; ++m) r[m] += -a.two_dx * (FR - ((m & 1) ? -FL : FL));
  } else {
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      const int dirn = f >> 1;          // 0: x-face, 1: y-face
      const bool upper = (f & 1) == 0;  // right / top
      const int fi = dirn == 0 ? ty * (TX + 1) + tx + (upper ? 1 : 0) : L::NFX + (ty + (upper ? 1 : 0)) * TX + tx;
      float h[N];
#pragma unroll
      for (int j = 0; j < N; ++j) h[j] = sF[fi * N + j];
      if (!upper && (dirn == 0 ? (a.perx || gi > 0) : (a.pery || gj > 0)))
        h[0] = fmaf(2.0f, law.flux_dev_dir(sc[hc + (dirn == 0 ? -1 : -HX)] - ubar, dirn), h[0]);
      // r[mx,my] -= 2/dx (hR[my] - (-1)^mx hL[my]) + 2/dy (hT[mx] - (-1)^my hB[mx])
      const float s2d = dirn == 0 ? a.two_dx : a.two_dy;
#pragma unroll
      for (int my = 0; my < N; ++my)
#pragma unroll
        for (int mx = 0; mx < N; ++mx) {
          const int nrm = dirn == 0 ? mx : my;  // mode index along the normal
          const float hv = dirn == 0 ? h[my] : h[mx];
          if (upper)
            r[mx + N * my] = fmaf(-s2d, hv, r[mx + N * my]);
          else
            r[mx + N * my] = fmaf(s2d, (nrm & 1) ? -hv : hv, r[mx + N * my]);
        }
    }
  }
}

// One tile of one stage: the whole path (a)-(e) for the cells [i0, i0+TX) x [j0, j0+TY)
// (SURR: the instantiation that also runs the surrogate sensor and the features mode; the
// plain instantiation carries none of that code, so its registers are unaffected)
// of the mesh described by a.  Every thread must have started the staging of the
// tabulations (stage_tables_to_smem) before the call: the tile's first cp.async wait and
// barrier complete it.  The function contains its own barriers and is called by every
// thread of the CTA.  A block of NB > TX * TY threads shares the loads, the vertices and
// the faces among all of them; its threads beyond the cells leave before the per-cell
// stages.
// TC: the tensor-core form of stage (c) (2D, p = 3, 8 x 16 tiles; TileLayout), with the
// CTA's TMEM allocation and MMA barrier in tcx; the TMEM is freed inside the tile.
template <int DIM, int P, int SYS, int TX, int TY, bool SURR = false, int NB = TX * TY, bool TC = false>
__device__ __forceinline__ void scalar_tile(const StageArgs& a, const DgTables<DIM, P>& T, int i0, int j0,
                                            float* smem, TcCtx tcx = {}) {
  using L = TileLayout<DIM, P, TX, TY, TC>;
  using Law = ScalarLaw<SYS, DIM>;
  constexpr int N = L::N, ND = L::ND, NT = L::NT;
  constexpr int HX = L::HX, NH = L::NH;
  constexpr int NY1 = DIM == 2 ? N : 1;  // tensor extent in y (1 in 1D)
  static_assert(!TC || (DIM == 2 && !SURR && NB == NT), "tensor-core form: plain 2D kernel, one thread per cell");
  float* sc = smem + L::OFF_SC;
  float* st = smem + (TC ? L::OFF_TSA : L::OFF_ST);
  float* sA = smem + L::OFF_A;
  float* sB = smem + L::OFF_B;
  float* sBd = smem + L::OFF_BD;
  float* sBk = smem + L::OFF_BK;
  float* sW = smem + L::OFF_W;
  float* sNq = smem + L::OFF_NQ;

  const int nx = a.nx, ny = DIM == 2 ? a.ny : 1;

  // ---- load tile + halo ---------------------------------------------------------------------
  // Asynchronous copies, every one of the thread's in flight before the first wait, landing
  // in a staging area (over the indicator and u_n regions, unused until later) and then
  // transposed to the mode-major layout sc[m][h]:
  //  - a cell of whole 16-byte chunks (Q1, Q3): 16-byte copies per cell, cell-major;
  //  - otherwise each halo row by stage_rows16, at the row's phase sph[r];
  //  - a state that is not 16-byte aligned: 4-byte copies straight into sc.
  static_assert(NH * ND <= L::STAGING, "halo staging must fit the indicator and u_n regions");
  constexpr int HY = L::HY, RSP = (HX * ND + 6) / 4 * 4;  // staging row stride (floats)
  static_assert(ND % 4 == 0 || HY * RSP <= L::STAGING, "halo row staging must fit the indicator and u_n regions");
  __shared__ int sph[HY];
  const bool aligned = (reinterpret_cast<uintptr_t>(a.u_in) & 15) == 0;
  const bool in16 = ND % 4 == 0 && aligned;
  const bool rows16 = ND % 4 != 0 && aligned;
  float* stg = smem + L::OFF_NQ;
  constexpr int NQ4 = ND / 4 > 0 ? ND / 4 : 1;  // used only where ND % 4 == 0
  if (rows16) {
    stage_rows16<ND, HX, HY, RSP, NB>(stg, sph, a.u_in, nx, DIM == 2 ? ny : 1, i0 - 1, DIM == 2 ? j0 - 1 : 0, a.perx,
                                      DIM == 2 && a.pery, a.status, CVW_EXTENT(a, lim_in));
  } else if (in16) {
    for (int f = threadIdx.x; f < NH * NQ4; f += NB) {
      const int h = f / NQ4, q = f - h * NQ4;
      const int r = DIM == 2 ? h / HX : 0, cc = h - r * HX;
      int gi = i0 - 1 + cc, gj = DIM == 2 ? j0 - 1 + r : 0;
      bool ok = true;
      if (gi < 0 || gi >= nx) {
        if (a.perx) gi = (gi + nx) % nx; else ok = false;
      }
      if (DIM == 2 && (gj < 0 || gj >= ny)) {
        if (a.pery) gj = (gj + ny) % ny; else ok = false;
      }
      ok = ok && CVW_SPAN(a.status, ((size_t)gj * nx + gi) * ND + 4 * q, 4, a.lim_in);
      cp_async16z(stg + 4 * f, ok ? a.u_in + ((size_t)gj * nx + gi) * ND + 4 * q : a.u_in, ok ? 16 : 0);
    }
  } else {
    for (int f = threadIdx.x; f < NH * ND; f += NB) {
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
      ok = ok && CVW_SPAN(a.status, ((size_t)gj * nx + gi) * ND + mm, 1, a.lim_in);
      cp_async4(sc + mm * NH + r * HX + cc, ok ? a.u_in + ((size_t)gj * nx + gi) * ND + mm : a.u_in, ok ? 4 : 0);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  if (in16) {
    for (int f = threadIdx.x; f < NH * NQ4; f += NB) {
      const int h = f / NQ4, q = f - h * NQ4;
      const float4 v = *reinterpret_cast<const float4*>(stg + 4 * f);
      sc[(4 * q + 0) * NH + h] = v.x;
      sc[(4 * q + 1) * NH + h] = v.y;
      sc[(4 * q + 2) * NH + h] = v.z;
      sc[(4 * q + 3) * NH + h] = v.w;
    }
    __syncthreads();
  } else if (rows16) {
    for (int h = threadIdx.x; h < NH; h += NB) {
      const int r = DIM == 2 ? h / HX : 0, cc = h - r * HX;
      const float* src = stg + r * RSP + sph[r] + cc * ND;
#pragma unroll
      for (int m = 0; m < ND; ++m) sc[m * NH + h] = src[m];
    }
    __syncthreads();
  }

  // u_n of the thread's own cell (RK stages 2 and 3), read only by the output: copied after
  // the halo burst so that it overlaps the stages below, and awaited before the output.
  // Only this thread reads u_n or writes u_out for its cell, so u_n may alias u_out.
  // Cell-major 16-byte copies where the cell is whole 16-byte chunks, else mode-major.
  const bool pre_un = (a.mode & kModeRK) && a.rk_a != 0.0f;
  const bool un16 = ND % 4 == 0 && (reinterpret_cast<uintptr_t>(a.u_n) & 15) == 0;
  {
    const int ogi = i0 + threadIdx.x % TX, ogj = DIM == 2 ? j0 + threadIdx.x / TX : 0;
    if (pre_un && threadIdx.x < NT && ogi < nx && ogj < ny &&
        CVW_SPAN(a.status, ((size_t)ogj * nx + ogi) * ND, ND, a.lim_in)) {
      const float* src = a.u_n + ((size_t)ogj * nx + ogi) * ND;
      float* sUn = smem + L::OFF_UN;
      if (un16) {
#pragma unroll
        for (int k = 0; k < ND / 4; ++k) cp_async16(sUn + threadIdx.x * ND + 4 * k, src + 4 * k);
      } else {
#pragma unroll 1
        for (int m = 0; m < ND; ++m) cp_async4(sUn + m * NT + threadIdx.x, src + m, 4);
      }
    }
  }

  // ---- (a)+(b): vertex candidates of the tile's vertices ------------------------------
  tile_vertex_phase<DIM, P, TX, TY, NB, TC>(a, T, sc, st, i0, j0, nx, ny);
  constexpr bool kSharedFaces = L::SHARED_FACES && !(SURR && P == 2);
  if constexpr (kSharedFaces) {
    if (!(a.mode & (kModeSensorOnly | kModeLimit | kModeFeatures)))
      tile_face_phase<DIM, P, SYS, TX, TY, NB>(a, sc, sB, sW, smem + L::OFF_F, i0, j0, nx, ny);
  }
  if constexpr (TC) tc::fence_proxy_async();  // the operand, for the tensor cores
  __syncthreads();
  if constexpr (TC) {
    if (threadIdx.x == 0) issue_corner_products<P, TX, TY>(smem, tcx);
  }
  pdl_launch_dependents();

  // ---- one thread per cell from here on (TC: one more barrier, after the sensor) -----------
  if (NB > NT && threadIdx.x >= NT) return;
  const int tx = threadIdx.x % TX, ty = DIM == 2 ? threadIdx.x / TX : 0;
  const int gi = i0 + tx, gj = DIM == 2 ? j0 + ty : 0;
  // (the checked build also checks the cell's span of u_out and its index in the per-cell
  // outputs)
  const bool active = gi < nx && gj < ny && CVW_SPAN(a.status, ((size_t)gj * nx + gi) * ND, ND, a.lim_out) &&
                      CVW_SPAN(a.status, (size_t)gj * nx + gi, 1, a.lim_cell);
  // the surrogate runs warp-wide on the tensor cores: cells outside the mesh take part
  // (on the tile's zero-filled halo data) and leave after it; so do they in the TC form,
  // whose TMEM loads are warp-collective
  bool use_mlp = false;
  if constexpr (DIM == 2 && SURR) use_mlp = a.mlp != nullptr && !(a.mode & (kModeLimit | kModeFeatures));
  if (!TC && !active && !use_mlp) return;
  const int hc = (DIM == 2 ? (ty + 1) * HX : 0) + tx + 1;
  const size_t cell = (size_t)gj * nx + gi;
  float c[ND];
#pragma unroll
  for (int m = 0; m < ND; ++m) c[m] = sc[m * NH + hc];
  float r[ND];  // the residual (TC: its faces' part is taken while the tensor cores run)
#pragma unroll
  for (int m = 0; m < ND; ++m) r[m] = 0.0f;

  // ---- (c) cell-vertex reconstruction and sensor --------------------------------------
  float n0;
  float wstar[L::NS];
  float gam;
  if constexpr (DIM == 2 && SURR) {
    if (a.mode & kModeFeatures) {
      gam = cell_sensor<DIM, P, TX, TY>(a, T, st, sA, c, tx, ty, n0, wstar);
      float f[kMlpIn];
      cell_features<P, TX, TY>(a, st, c[0], n0, tx, ty, f);
#pragma unroll
      for (int j = 0; j < kMlpIn; ++j) a.feat_out[cell * kMlpIn + j] = f[j];
      if (a.gamma_out) a.gamma_out[cell] = gam;
      if (a.norm_out) a.norm_out[cell] = n0;
      return;
    }
    if (use_mlp) {
      n0 = cell_norm0<DIM, P>(T, c);
      float f[kMlpIn];
      cell_features<P, TX, TY>(a, st, c[0], n0, tx, ty, f);
      float o0 = 0.0f, o1 = 0.0f;
      const bool live = active && n0 > kNearFlat * (fabsf(c[0]) + 1.0f);
      const int warp = threadIdx.x >> 5;
      // a warp whose cells are all flat to rounding (S7) skips the network
      if (__any_sync(0xffffffffu, live))
        mlp_warp(*reinterpret_cast<const MlpPacked*>(smem + L::OFF_MLP), f,
                 reinterpret_cast<__nv_bfloat16*>(smem + L::OFF_XS) + warp * 32 * 16, o0, o1);
      if (!active) return;
      const float conf = 1.0f / (1.0f + __expf(-o1));
      const bool fallback = live && !(conf >= a.mlp_conf_min);
      if (a.mlp_fallbacks) {  // one atomic per warp: the count of its falling-back cells
        const unsigned am = __activemask(), fm = __ballot_sync(am, fallback);
        if (fm && (threadIdx.x & 31) == (unsigned)(__ffs(am) - 1)) atomicAdd(a.mlp_fallbacks, (unsigned)__popc(fm));
      }
      if (!live) {
        gam = 1.0f;  // flat to rounding (readings A7, S7): no network, no fallback
      } else if (!fallback) {
        gam = 1.0f / (1.0f + __expf(-o0));
      } else {
        gam = cell_sensor<DIM, P, TX, TY>(a, T, st, sA, c, tx, ty, n0, wstar);
      }
      if (a.sensor_mode == CVWENO_SENSOR_SMOOTH) gam = 1.0f;
      if (a.sensor_mode == CVWENO_SENSOR_TROUBLED) gam = 0.0f;
    } else {
      gam = cell_sensor<DIM, P, TX, TY>(a, T, st, sA, c, tx, ty, n0, wstar);
    }
  } else if constexpr (TC) {
    const bool faces_now = active && !(a.mode & (kModeSensorOnly | kModeLimit));
    gam = cell_sensor_tc<DIM, P, TX, TY>(a, T, tcx, c, n0, wstar, [&] {
      if (faces_now) shared_face_residual<DIM, P, SYS, TX, TY, TC>(a, Law(a, c[0]), smem, sc, c[0], tx, ty, gi, gj, hc, r);
    });
    if (!active) return;
  } else {
    gam = cell_sensor<DIM, P, TX, TY>(a, T, st, sA, c, tx, ty, n0, wstar);
  }

  // ---- HWENO limiter (Sec. 3): u^{e,*} = mean of u^e + R^{-1} w* on the other modes ----
  if (a.mode & kModeLimit) {
    const bool lim = a.limit_all || (gam < a.c_gamma && n0 > 1e-30f);
    float* o = a.u_out + cell * ND;
    if (!lim) {
#pragma unroll
      for (int m = 0; m < ND; ++m) o[m] = c[m];
    } else {
      constexpr int NS = L::NS;
      float x[NS];
#pragma unroll
      for (int i = NS - 1; i >= 0; --i) {  // back substitution with the upper-triangular R
        float acc = wstar[i];
#pragma unroll
        for (int j = i + 1; j < NS; ++j) acc = fmaf(-T.R[i][j], x[j], acc);
        x[i] = acc / T.R[i][i];
      }
      o[0] = c[0];
      bool bad = !isfinite(c[0]);
#pragma unroll
      for (int i = 0; i < NS; ++i) {
        o[i + 1] = x[i];
        bad |= !isfinite(x[i]);
      }
      if (bad) atomicOr(a.status, kStatNonfinite);
    }
    if (a.troubled_out) a.troubled_out[cell] = lim ? 1 : 0;
    return;
  }

  // ---- own trace polynomials along each face, as deviations from the mean -------------------
  // u(x) = ubar + (non-mean modes): rounding stays relative to the in-cell variation.
  const float ubar = c[0];
  const Law law(a, ubar);
  constexpr int NF = DIM == 2 ? N : 1;  // nodes per face
  float trR[N], trL[N], trT[N], trB[N];
  if constexpr (DIM == 1) {
    float sR = 0.0f, sL = 0.0f;
#pragma unroll
    for (int m = 1; m < N; ++m) {
      sR += c[m];
      sL += (m & 1) ? -c[m] : c[m];
    }
    trR[0] = sR;
    trL[0] = sL;
  } else {
#pragma unroll
    for (int j = 0; j < N; ++j) {
      float r = 0.0f, l = 0.0f, t = 0.0f, b = 0.0f;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const float cr = (i + N * j) ? c[i + N * j] : 0.0f, ct = (j + N * i) ? c[j + N * i] : 0.0f;
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
  }

  // ---- lambda_e (over face and volume nodes) and (d) the SC weights ------------------------------
  bool troubled = false;
  float afac = -1.0f;  // alpha_q = Nq[q] * afac where afac >= 0, else alpha_q = 1
  float lam = a.lambda_const > 0.0f ? a.lambda_const : 0.0f;
  if (!(a.lambda_const > 0.0f)) {
#pragma unroll 1
    for (int q = 0; q < NF; ++q) {
      float vr = trR[0], vl = trL[0], vt = 0.0f, vbb = 0.0f;
      if constexpr (DIM == 2) {
        vr = vl = 0.0f;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const float bq = sB[q * N + j];
          vr = fmaf(bq, trR[j], vr);
          vl = fmaf(bq, trL[j], vl);
          vt = fmaf(bq, trT[j], vt);
          vbb = fmaf(bq, trB[j], vbb);
        }
      }
      lam = fmaxf(lam, fmaxf(law.speed(ubar + vr), law.speed(ubar + vl)));
      if constexpr (DIM == 2) lam = fmaxf(lam, fmaxf(law.speed(ubar + vt), law.speed(ubar + vbb)));
    }
  }
  if (!(a.mode & kModeSensorOnly)) {
    troubled = a.sc && gam < a.c_gamma && n0 > 1e-30f;
    if (a.troubled_override) {
      int ov = a.troubled_override[cell];
      if (ov >= 0) troubled = ov && n0 > 1e-30f;
    }
  }
  const bool need_sc = troubled && gam < 1.0f;
  if (!(a.lambda_const > 0.0f) || need_sc) {
    float s1 = 0.0f, s2 = 0.0f;
#pragma unroll (DIM == 1 || P == 1 ? N : 1)
    for (int qx = 0; qx < N; ++qx) {
      float tb[NY1], td[NY1];
#pragma unroll
      for (int my = 0; my < NY1; ++my) {
        float s0 = 0.0f, sd = 0.0f;
#pragma unroll
        for (int mx = 0; mx < N; ++mx) {
          const float cm = (mx + N * my) ? c[mx + N * my] : 0.0f;
          s0 = fmaf(sB[qx * N + mx], cm, s0);
          sd = fmaf(sBd[qx * N + mx], cm, sd);
        }
        tb[my] = s0;
        td[my] = sd;
      }
      float X[N][NY1];  // [kx][my]: x-derivatives of order kx at xi_qx (stage d only)
      if (need_sc) {
#pragma unroll
        for (int kx = 0; kx < N; ++kx)
#pragma unroll
          for (int my = 0; my < NY1; ++my) {
            float acc = 0.0f;
#pragma unroll
            for (int mx = 0; mx < N; ++mx) acc = fmaf(sBk[(kx * N + qx) * N + mx], c[mx + N * my], acc);
            X[kx][my] = acc;
          }
      }
#pragma unroll 1
      for (int qy = 0; qy < NY1; ++qy) {
        float du = tb[0], ux = td[0], uy = 0.0f;
        if constexpr (DIM == 2) {
          du = ux = 0.0f;
#pragma unroll
          for (int my = 0; my < N; ++my) {
            const float bq = sB[qy * N + my], dq = sBd[qy * N + my];
            du = fmaf(bq, tb[my], du);
            ux = fmaf(bq, td[my], ux);
            uy = fmaf(dq, tb[my], uy);
          }
        }
        if (!(a.lambda_const > 0.0f)) lam = fmaxf(lam, law.speed(ubar + du));
        if (need_sc) {
          float n2 = 0.0f;
#pragma unroll
          for (int ky = 0; ky < NY1; ++ky)
#pragma unroll
            for (int kx = 0; kx < N; ++kx) {
              if (kx + ky == 0) continue;
              float dk = X[kx][0];
              if constexpr (DIM == 2) {
                dk = 0.0f;
#pragma unroll
                for (int my = 0; my < N; ++my) dk = fmaf(sBk[(ky * N + qy) * N + my], X[kx][my], dk);
              }
              n2 = fmaf(T.sigma[kx + N * ky] * dk, dk, n2);
            }
          const float nq = sqrtf(n2);
          sNq[(qx + N * qy) * NT + threadIdx.x] = nq;
          const float gx = a.two_dx * ux, gy = a.two_dy * uy;
          const float g = fmaf(gx, gx, gy * gy);
          const float W = sW[qx] * (DIM == 2 ? sW[qy] : 1.0f);
          s1 = fmaf(W, g, s1);
          s2 = fmaf(W * nq, g, s2);
        }
      }
    }
    if (need_sc && s2 > 0.0f) afac = s1 / s2;
  }
  const float nu = lam * a.nu_scale;
  if (a.gamma_out) a.gamma_out[cell] = gam;
  if (a.nu_out) a.nu_out[cell] = nu;
  if (a.lambda_out) a.lambda_out[cell] = lam;
  if (a.mode & kModeSensorOnly) return;
  if (a.troubled_out) a.troubled_out[cell] = troubled ? 1 : 0;
  if (a.alpha_out) {
#pragma unroll 1
    for (int q = 0; q < ND; ++q) a.alpha_out[cell * ND + q] = afac >= 0.0f ? sNq[q * NT + threadIdx.x] * afac : 1.0f;
  }

  // ---- (e) residual, deviation form ----------------------------------------------------------
  const float mu = (1.0f - gam) * nu;
  if constexpr (kSharedFaces) {
    if constexpr (!TC) shared_face_residual<DIM, P, SYS, TX, TY, TC>(a, law, smem, sc, ubar, tx, ty, gi, gj, hc, r);
  } else {
    // faces: neighbour traces relative to this cell's mean (ghost = own trace on a
    // transmissive side)
    if constexpr (DIM == 1) {
      const bool hasR = a.perx || gi + 1 < nx, hasL = a.perx || gi > 0;
      float nbR = trR[0], nbL = trL[0];
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
      const float FR = llf_dev(law, a, ubar, trR[0], nbR, 0);
      const float FL = llf_dev(law, a, ubar, nbL, trL[0], 0);
  #pragma unroll
      for (int m = 0; m < N; ++m) r[m] = -a.two_dx * (FR - ((m & 1) ? -FL : FL));
    } else {
      // face f: 0 right (+x), 1 left, 2 top (+y), 3 bottom.  The neighbour's trace along
      // the shared face relative to ubar, a rolled loop over the face nodes, and the
      // projection onto the tangential modes h[j] = sum_q w_q P_j(xi_q) F_q.
  #pragma unroll
      for (int f = 0; f < 4; ++f) {
        const int dirn = f >> 1;          // 0: x-face, 1: y-face
        const bool upper = (f & 1) == 0;  // right / top
        const int off = dirn == 0 ? (upper ? 1 : -1) : (upper ? HX : -HX);
        const bool has = dirn == 0 ? (a.perx || (upper ? gi + 1 < nx : gi > 0))
                                   : (a.pery || (upper ? gj + 1 < ny : gj > 0));
        const float* own = dirn == 0 ? (upper ? trR : trL) : (upper ? trT : trB);
        float nb[N];
  #pragma unroll
        for (int j = 0; j < N; ++j) {
          float s = 0.0f;
  #pragma unroll
          for (int i = 0; i < N; ++i) {
            const int m = dirn == 0 ? i + N * j : j + N * i;
            if (m == 0) continue;
            const float v = sc[m * NH + hc + off];
            // the neighbour meets this face with its opposite side: sign (-1)^i on a
            // right/top face (its left/bottom side), +1 on a left/bottom face
            s += (upper && (i & 1)) ? -v : v;
          }
          nb[j] = s;
        }
        const float dmean = has ? sc[hc + off] - ubar : 0.0f;
        float h[N];
  #pragma unroll
        for (int j = 0; j < N; ++j) h[j] = 0.0f;
  #pragma unroll 1
        for (int q = 0; q < N; ++q) {
          float vo = 0.0f, vn = 0.0f;
  #pragma unroll
          for (int j = 0; j < N; ++j) {
            const float bq = sB[q * N + j];
            vo = fmaf(bq, own[j], vo);
            vn = fmaf(bq, nb[j], vn);
          }
          vn = has ? dmean + vn : vo;
          const float F = upper ? llf_dev(law, a, ubar, vo, vn, dirn) : llf_dev(law, a, ubar, vn, vo, dirn);
          const float wq = sW[q] * F;
  #pragma unroll
          for (int j = 0; j < N; ++j) h[j] = fmaf(wq, sB[q * N + j], h[j]);
        }
        // r[mx,my] -= 2/dx (hR[my] - (-1)^mx hL[my]) + 2/dy (hT[mx] - (-1)^my hB[mx])
        const float s2d = dirn == 0 ? a.two_dx : a.two_dy;
  #pragma unroll
        for (int my = 0; my < N; ++my)
  #pragma unroll
          for (int mx = 0; mx < N; ++mx) {
            const int nrm = dirn == 0 ? mx : my;  // mode index along the normal
            const float hv = dirn == 0 ? h[my] : h[mx];
            if (upper)
              r[mx + N * my] = fmaf(-s2d, hv, r[mx + N * my]);
            else
              r[mx + N * my] = fmaf(s2d, (nrm & 1) ? -hv : hv, r[mx + N * my]);
          }
      }
    }
  }
  // volume: flux deviation and alpha-weighted viscous term, projected by sum factorisation
#pragma unroll (DIM == 1 || P == 1 ? N : 1)
  for (int qx = 0; qx < N; ++qx) {
    float tb[NY1], td[NY1];
#pragma unroll
    for (int my = 0; my < NY1; ++my) {
      float s0 = 0.0f, sd = 0.0f;
#pragma unroll
      for (int mx = 0; mx < N; ++mx) {
        const float cm = (mx + N * my) ? c[mx + N * my] : 0.0f;
        s0 = fmaf(sB[qx * N + mx], cm, s0);
        sd = fmaf(sBd[qx * N + mx], cm, sd);
      }
      tb[my] = s0;
      td[my] = sd;
    }
    float hx[NY1], hy[NY1];
#pragma unroll
    for (int my = 0; my < NY1; ++my) hx[my] = hy[my] = 0.0f;
    const float wx = sW[qx];
#pragma unroll 1
    for (int qy = 0; qy < NY1; ++qy) {
      float du = tb[0], ux = td[0], uy = 0.0f;
      if constexpr (DIM == 2) {
        du = ux = 0.0f;
#pragma unroll
        for (int my = 0; my < N; ++my) {
          const float bq = sB[qy * N + my], dq = sBd[qy * N + my];
          du = fmaf(bq, tb[my], du);
          ux = fmaf(bq, td[my], ux);
          uy = fmaf(dq, tb[my], uy);
        }
      }
      float fx, fy;
      law.flux_dev(du, fx, fy);
      const float al = afac >= 0.0f ? sNq[(qx + N * qy) * NT + threadIdx.x] * afac : 1.0f;
      const float W = DIM == 2 ? wx * sW[qy] : wx;
      const float gx = W * (fx - mu * al * a.two_dx * ux);
      if constexpr (DIM == 2) {
        const float gy = W * (fy - mu * al * a.two_dy * uy);
#pragma unroll
        for (int my = 0; my < N; ++my) {
          hx[my] = fmaf(sB[qy * N + my], gx, hx[my]);
          hy[my] = fmaf(sBd[qy * N + my], gy, hy[my]);
        }
      } else {
        hx[0] = gx;
      }
    }
#pragma unroll
    for (int my = 0; my < NY1; ++my)
#pragma unroll
      for (int mx = 0; mx < N; ++mx) {
        if (mx + my == 0) continue;
        float v = r[mx + N * my];
        v = fmaf(a.two_dx * sBd[qx * N + mx], hx[my], v);
        if constexpr (DIM == 2) v = fmaf(a.two_dy * sB[qx * N + mx], hy[my], v);
        r[mx + N * my] = v;
      }
  }
  // M^{-1} and output (into r); 16-byte stores where the cell is whole 16-byte chunks and
  // the output is 16-byte aligned
  bool bad = false;
  float* out = a.u_out + cell * ND;
  const float* sUn = smem + L::OFF_UN;  // u_n of this cell
  if (pre_un) cp_async_wait_all();
#pragma unroll
  for (int m = 0; m < ND; ++m) {
    const int mx = m % N, my = DIM == 2 ? m / N : 0;
    const float minv = DIM == 2 ? 0.25f * (2 * mx + 1) * (2 * my + 1) : 0.5f * (2 * mx + 1);
    float d = r[m] * minv;
    bad |= !isfinite(d);
    if (a.mode & kModeRK) {
      float v = fmaf(a.dt, d, c[m]);
      if (pre_un) {
        const float un = un16 ? sUn[threadIdx.x * ND + m] : sUn[m * NT + threadIdx.x];
        v = fmaf(a.rk_b, v - un, un);
      }
      d = v;
    }
    r[m] = d;
  }
  if (ND % 4 == 0 && (reinterpret_cast<uintptr_t>(a.u_out) & 15) == 0) {
#pragma unroll
    for (int q = 0; q < ND / 4; ++q)
      reinterpret_cast<float4*>(out)[q] = make_float4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
  } else {
#pragma unroll
    for (int m = 0; m < ND; ++m) out[m] = r[m];
  }
  if (bad) atomicOr(a.status, kStatNonfinite);
}

template <int DIM, int P, int SYS, int TX, int TY, bool SURR, int NB = TX * TY, bool TC = false>
__device__ __forceinline__ void stage_body(const StageArgs& a, const DgTables<DIM, P>& T) {
  extern __shared__ __align__(16) float smem[];
  TcCtx tcx = {};
  if constexpr (TC) {
    // published by the tile's first barrier (after its loads)
    __shared__ uint32_t tmem_slot, tc_done;
    __shared__ uint64_t mma_bar;
    if (threadIdx.x < 32) {
      tc::tmem_alloc(&tmem_slot, kTcCols);
      tc::fence_before();
    }
    if (threadIdx.x == 0) {
      tc::mbar_init(&mma_bar, 1);
      tc_done = 0;
    }
    tcx = TcCtx{&tmem_slot, tc::smem_u32(&mma_bar), &tc_done};
  }
  stage_tables_to_smem<DIM, P, TX, TY, NB, TC>(a.tab_img, smem);  // lands with the tile's first wait
  pdl_wait();  // everything below reads or writes what earlier kernels write
  if constexpr (SURR && DIM == 2) {
    if (a.mlp) stage_mlp_to_smem<DIM, P, TX, TY, NB>(a.mlp, smem);
  }
  scalar_tile<DIM, P, SYS, TX, TY, SURR, NB, TC>(a, T, blockIdx.x * TX, DIM == 2 ? blockIdx.y * TY : 0, smem, tcx);
}

// Threads of a block of the plain stage kernel.  One warp more than the tile's cells in 1D
// and below p = 3 in 2D, so that the tile's (TX + 1) (TY + 1) vertices take one round,
// and the faces beside them fewer.  At p >= 3 the extra warp's registers would cost a
// resident CTA per SM.
template <int DIM, int P, int TX, int TY>
__host__ __device__ constexpr int stage_block_threads() {
  return DIM == 1 || P <= 2 ? TX * TY + 32 : TX * TY;
}

template <int DIM, int P, int SYS, int TX, int TY>
__global__ void __launch_bounds__(stage_block_threads<DIM, P, TX, TY>())
    dg_scalar_stage(const __grid_constant__ StageArgs a, const __grid_constant__ DgTables<DIM, P> T) {
  stage_body<DIM, P, SYS, TX, TY, false, stage_block_threads<DIM, P, TX, TY>()>(a, T);
}

// The tensor-core form of the 2D Q3 stage kernel: 8 x 16 tiles, the sensor's corner
// products on tcgen05 in split TF32 (TileLayout, issue_corner_products); 4 CTAs per SM.
template <int SYS>
__global__ void __launch_bounds__(128, 4)
    dg_scalar_stage_tc(const __grid_constant__ StageArgs a, const __grid_constant__ DgTables<2, 3> T) {
  stage_body<2, 3, SYS, 8, 16, false, 128, true>(a, T);
}

// nsteps SSP-RK3 steps of a 1D mesh that is a single tile (nx <= TX), in one launch.  The
// halo of a stage is this block's own output of the stage before, so a block barrier
// (which orders the block's global writes before its later reads) stands in for the
// kernel boundary; the tabulations are staged once.  Each stage is the stage kernel's
// code with the same block, so the results are bitwise those of three launches per step.
template <int P, int SYS, int TX>
__global__ void __launch_bounds__(stage_block_threads<1, P, TX, 1>())
    dg_scalar_steps_tile(const __grid_constant__ StepArgs s, const __grid_constant__ DgTables<1, P> T) {
  constexpr int NB = stage_block_threads<1, P, TX, 1>();
  extern __shared__ __align__(16) float smem[];
  stage_tables_to_smem<1, P, TX, 1, NB>(s.st[0].tab_img, smem);
  pdl_wait();
#pragma unroll 1
  for (int n = 0; n < s.nsteps; ++n) {
    scalar_tile<1, P, SYS, TX, 1, false, NB>(s.st[0], T, 0, 0, smem);
    __syncthreads();
    scalar_tile<1, P, SYS, TX, 1, false, NB>(s.st[1], T, 0, 0, smem);
    __syncthreads();
    scalar_tile<1, P, SYS, TX, 1, false, NB>(s.st[2], T, 0, 0, smem);
    __syncthreads();
  }
}

// The surrogate instantiation takes the plain kernel's block and is held to the register
// budget of 4 resident CTAs up to p = 3 and 3 at p = 4, which the network's fragments
// would otherwise exceed.
template <int DIM, int P, int SYS, int TX, int TY>
__global__ void __launch_bounds__(stage_block_threads<DIM, P, TX, TY>(), (P >= 4 ? 3 : 4) * (128 / (TX * TY)))
    dg_scalar_stage_surrogate(const __grid_constant__ StageArgs a, const __grid_constant__ DgTables<DIM, P> T) {
  stage_body<DIM, P, SYS, TX, TY, true, stage_block_threads<DIM, P, TX, TY>()>(a, T);
}

}  // namespace cvw
