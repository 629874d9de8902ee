// Continuous Galerkin (CG) stage for scalar conservation laws on periodic meshes.
//
// State: values at the Gauss-Lobatto-Legendre nodes of the global lattice
// (p nx) x (p ny), node I + (p nx) J.  One RK stage is
//   K1 cg_stage_cells   tile of cells + one-cell halo: nodal -> Legendre modes, the same
//                       vertex phase and cell sensor as DG (stages a-c), the lumped-mass
//                       projection P_h grad u at the cell's own nodes (reading A13, from
//                       the local integrals of the tile and halo cells), the CG SC weights
//                       with f_q = |grad u|^2 - gamma grad u . P_h grad u (Sec. 4; A24),
//                       and the cell-local residual
//                       int grad phi . f(u) - nu_e sum_q alpha_q w_q grad phi . (grad u - gamma P_h grad u)
//                       (Sec. 2.2, CG form of eq. stab)
//   K2 cg_node_stage2d  (2D) per tile of lattice nodes: the deterministic nodal assembly
//                       r_j, du = r_j / ML_j, and the two defect-correction sweeps
//                       du <- du + ML^{-1}(r - M_C du) (reading A12) with the
//                       tensor-product consistent mass, the second writing the SSP-RK3
//                       combination (or du itself for a residual); r and the first
//                       iterate are formed on a halo of 2p nodes, so one launch suffices
//   1D: cg_node_rhs (assembly, du = r / ML) and two cg_node_sweep launches
// Nodal sums gather the cells around a node in a fixed order.
#include "dg_scalar_kernel.cuh"

namespace cvw {
namespace {

// i mod n for any int i (n > 0), without a division when i is already in range
__device__ __forceinline__ int wrap_index(int i, int n) {
  if ((unsigned)i < (unsigned)n) return i;
  i %= n;
  return i < 0 ? i + n : i;
}

template <int DIM, int P, int TX, int TY>
struct CgLayout {
  using L = TileLayout<DIM, P, TX, TY>;
  static constexpr int N = P + 1, ND = L::ND, NH = L::NH;
  static constexpr int NNX = P * (TX + 2) + 1, NNY = DIM == 2 ? P * (TY + 2) + 1 : 1;
  // nodal rows at a 16-byte stride with room for a per-row phase of up to 3 floats
  static constexpr int NNXP = (NNX + 3 + 3) / 4 * 4;
  // The nodal tile is dead once the halo cells are converted to modes, and the local
  // integrals are written after that barrier: both start at the u_n region of the DG
  // layout, which the CG kernel does not use (its RK combination runs on the nodes).
  static constexpr int OFF_NODE = L::OFF_UN;              // [NNY][NNXP] nodal values
  static constexpr int OFF_BX = L::OFF_UN;                // [ND][NH] int phi_a d_x u
  static constexpr int OFF_BY = OFF_BX + ND * NH;         // [ND][NH] int phi_a d_y u
  static constexpr int FLOATS = L::OFF_UN + (2 * ND * NH > NNXP * NNY ? 2 * ND * NH : NNXP * NNY);
  static constexpr size_t BYTES = sizeof(float) * (size_t)FLOATS;
};

// lumped mass of a 1D lattice node with local index a in [0, p): its GLL weight times
// dx/2, counted twice at cell vertices (two cells share them)
template <int DIM, int P>
__device__ __forceinline__ float ml1(const CgTables<DIM, P>& C, int a, float h) {
  return (a == 0 ? 2.0f : 1.0f) * C.wl[a] * h;
}

// Threads of a block of the CG cell kernel: one warp more than the tile's cells in 1D and
// at p = 1, so that the tile's (TX + 1) (TY + 1) vertices take one round and the halo
// ring's integrals fall on the extra warp (KPP 256^2 CG Q1: 0.0411 -> 0.0391 ms per step;
// at p = 2 the same block was 19 % slower).
template <int DIM, int P, int TX, int TY>
__host__ __device__ constexpr int cg_block_threads() {
  return DIM == 1 || P == 1 ? TX * TY + 32 : TX * TY;
}

template <int DIM, int P, int SYS, int TX, int TY>
__global__ void __launch_bounds__(cg_block_threads<DIM, P, TX, TY>()) cg_stage_cells(const __grid_constant__ StageArgs a,
                                                          const __grid_constant__ DgTables<DIM, P> T,
                                                          const __grid_constant__ CgTables<DIM, P> C) {
  using L = TileLayout<DIM, P, TX, TY>;
  using G = CgLayout<DIM, P, TX, TY>;
  using Law = ScalarLaw<SYS, DIM>;
  constexpr int N = L::N, ND = L::ND, NT = L::NT, HX = L::HX, NH = L::NH;
  constexpr int NB = cg_block_threads<DIM, P, TX, TY>();  // threads of the block
  constexpr int NNX = G::NNX, NNY = G::NNY, NNXP = G::NNXP;
  constexpr int NY1 = DIM == 2 ? N : 1;
  extern __shared__ __align__(16) float smem[];
  float* sc = smem + L::OFF_SC;
  float* st = smem + L::OFF_ST;
  const float* sA = smem + L::OFF_A;
  const float* sB = smem + L::OFF_B;
  const float* sBd = smem + L::OFF_BD;
  const float* sBk = smem + L::OFF_BK;
  const float* sW = smem + L::OFF_W;
  float* sNq = smem + L::OFF_NQ;
  float* snode = smem + G::OFF_NODE;
  float* sbx = smem + G::OFF_BX;
  float* sby = smem + G::OFF_BY;

  const int nx = a.nx, ny = DIM == 2 ? a.ny : 1;
  const int nnx = a.nnx, nny = DIM == 2 ? a.nny : 1;
  const int i0 = blockIdx.x * TX, j0 = DIM == 2 ? blockIdx.y * TY : 0;
  const float hdx = 1.0f / a.two_dx, hdy = DIM == 2 ? 1.0f / a.two_dy : 1.0f;

  // ---- nodal values of the tile and its halo (periodic lattice) -------------------------
  stage_tables_to_smem<DIM, P, TX, TY, NB>(a.tab_img, smem);
  pdl_wait();  // everything below reads or writes what earlier kernels write
  // Node (ix, iy) lands at snode[iy][sph[iy] + ix].  Where the tile's rows do not wrap in x
  // and the state is 16-byte aligned, each row is copied as the 16-byte chunks that cover
  // it: the first chunk starts up to 3 floats early (sph, the row's phase), the last is
  // zero-filled past the row's last node, so no read leaves the row's own span or the
  // floats just before it.  Otherwise 4-byte copies, phase 0.
  __shared__ int sph[NNY];
  {
    const int I0 = P * (i0 - 1), J0 = DIM == 2 ? P * (j0 - 1) : 0;
    const bool rows16 = I0 >= 0 && I0 + NNX <= nnx && (reinterpret_cast<uintptr_t>(a.u_in) & 15) == 0;
    if (rows16) {
      constexpr int NCH = NNXP / 4;  // chunks per row
      for (int f = threadIdx.x; f < NNY * NCH; f += NB) {
        const int iy = f / NCH, k = f - iy * NCH;
        const int J = DIM == 2 ? wrap_index(J0 + iy, nny) : 0;
        const int64_t g0 = (int64_t)J * nnx + I0;  // the row's first node
        const int ph = (int)(g0 & 3);
        const int64_t c0 = g0 - ph + 4 * k;
        const int64_t left = g0 + NNX - c0;  // wanted floats from the chunk's start on
        if (left > 0 && CVW_SPAN(a.status, c0, left >= 4 ? 4 : left, a.lim_in))
          cp_async16z(snode + iy * NNXP + 4 * k, a.u_in + c0, left >= 4 ? 16 : (int)left * 4);
        if (k == 0) sph[iy] = ph;
      }
    } else {
      for (int f = threadIdx.x; f < NNX * NNY; f += NB) {
        const int ix = f % NNX, iy = f / NNX;
        const int I = wrap_index(I0 + ix, nnx);
        const int J = DIM == 2 ? wrap_index(J0 + iy, nny) : 0;
        if (CVW_SPAN(a.status, (size_t)J * nnx + I, 1, a.lim_in)) cp_async4(snode + iy * NNXP + ix, a.u_in + (size_t)J * nnx + I, 4);
      }
      for (int iy = threadIdx.x; iy < NNY; iy += NB) sph[iy] = 0;
    }
  }
  cp_async_wait_all();
  __syncthreads();
  // ---- every halo cell: nodal -> Legendre modes c = (V x V) u_loc -------------------------
  // The transform is applied to u_loc - u_ref (u_ref = the cell's first node): every mode
  // but the mean is unchanged (the rows of V beyond the mean sum to zero), the mean gets
  // u_ref back, and a constant cell yields exactly zero non-mean modes.
  for (int h = threadIdx.x; h < NH; h += NB) {
    const int hx = h % HX, hy = DIM == 2 ? h / HX : 0;
    float ul[ND];
#pragma unroll
    for (int b = 0; b < NY1; ++b)
#pragma unroll
      for (int aa = 0; aa < N; ++aa) ul[aa + N * b] = snode[sph[P * hy + b] + (P * hx + aa) + NNXP * (P * hy + b)];
    const float uref = ul[0];
#pragma unroll
    for (int m = 0; m < ND; ++m) ul[m] -= uref;
    float tmp[N][NY1];  // [mx][b]
#pragma unroll
    for (int mx = 0; mx < N; ++mx)
#pragma unroll
      for (int b = 0; b < NY1; ++b) {
        float acc = 0.0f;
#pragma unroll
        for (int aa = 0; aa < N; ++aa) acc = fmaf(C.V[mx][aa], ul[aa + N * b], acc);
        tmp[mx][b] = acc;
      }
#pragma unroll
    for (int my = 0; my < NY1; ++my)
#pragma unroll
      for (int mx = 0; mx < N; ++mx) {
        float acc = tmp[mx][0];
        if constexpr (DIM == 2) {
          acc = 0.0f;
#pragma unroll
          for (int b = 0; b < N; ++b) acc = fmaf(C.V[my][b], tmp[mx][b], acc);
        }
        sc[(mx + N * my) * NH + h] = (mx + my == 0) ? acc + uref : acc;
      }
  }
  __syncthreads();
  // ---- (a)+(b) vertex candidates (shared with DG) ---------------------------------------
  tile_vertex_phase<DIM, P, TX, TY, NB>(a, T, sc, st, i0, j0, nx, ny);
  // ---- P_h local integrals b_a = int phi_a grad u (reading A13) ------------------------------
  // For u = sum_m c_m P_mx P_my on the cell, with dx dy / 4 = hdx hdy and the factor 2/dx
  // of d/dx cancelling hdx (Em, Dm: integrals of l_a against P_m and P_m'):
  //   bx[a,b] = hdy sum_{mx,my} Dm[a][mx] Em[b][my] c[mx,my]
  //   by[a,b] = hdx sum_{mx,my} Em[a][mx] Dm[b][my] c[mx,my]
  // A tile cell takes every entry; a halo cell only those of its nodes on the tile's
  // boundary, the ones that the tile's nodes gather (one row or column of nodes).
  if constexpr (DIM == 1) {
    for (int h = threadIdx.x; h < NH; h += NB) {
#pragma unroll
      for (int aa = 0; aa < N; ++aa) {
        float acc = 0.0f;
#pragma unroll
        for (int m = 0; m < N; ++m) acc = fmaf(C.Dm[aa][m], sc[m * NH + h], acc);
        sbx[aa * NH + h] = acc;
        sby[aa * NH + h] = 0.0f;
      }
    }
  } else {
    constexpr int HY = L::HY;
    if (threadIdx.x < NT) {
      const int h = (threadIdx.x / TX + 1) * HX + threadIdx.x % TX + 1;
      float c[ND];
#pragma unroll
      for (int m = 0; m < ND; ++m) c[m] = sc[m * NH + h];
      float tE[N][N], tD[N][N];  // [b][mx]: the y-contractions
#pragma unroll
      for (int b = 0; b < N; ++b)
#pragma unroll
        for (int mx = 0; mx < N; ++mx) {
          float e = 0.0f, d = 0.0f;
#pragma unroll
          for (int my = 0; my < N; ++my) {
            e = fmaf(C.Em[b][my], c[mx + N * my], e);
            d = fmaf(C.Dm[b][my], c[mx + N * my], d);
          }
          tE[b][mx] = e;
          tD[b][mx] = d;
        }
#pragma unroll
      for (int b = 0; b < N; ++b)
#pragma unroll
        for (int aa = 0; aa < N; ++aa) {
          float bx = 0.0f, by = 0.0f;
#pragma unroll
          for (int mx = 0; mx < N; ++mx) {
            bx = fmaf(C.Dm[aa][mx], tE[b][mx], bx);
            by = fmaf(C.Em[aa][mx], tD[b][mx], by);
          }
          sbx[(aa + N * b) * NH + h] = hdy * bx;
          sby[(aa + N * b) * NH + h] = hdx * by;
        }
    }
    // halo ring: the bottom and top rows (corners included) need the node row b = l that
    // faces the tile (l = P below it, 0 above), the left and right columns the node
    // column a = l (P left of it, 0 right)
    constexpr int NR = 2 * HX + 2 * TY;
    // from the block's last thread backwards: the vertex phase's extra round (if any) falls
    // on the first warp, the ring on the last ones
    for (int r = NB - 1 - threadIdx.x; r < NR; r += NB) {
      const bool row = r < 2 * HX;
      int hx, hy, l;
      if (row) {
        const bool top = r >= HX;
        hx = top ? r - HX : r;
        hy = top ? HY - 1 : 0;
        l = top ? 0 : P;
      } else {
        const int rr = r - 2 * HX;
        const bool right = rr >= TY;
        hx = right ? HX - 1 : 0;
        hy = 1 + (right ? rr - TY : rr);
        l = right ? 0 : P;
      }
      const int h = hy * HX + hx;
      float c[ND];
#pragma unroll
      for (int m = 0; m < ND; ++m) c[m] = sc[m * NH + h];
      // s1: the contraction along the fixed direction with Em (row) or Dm (column) of
      // node l; s2 with the other table
      float s1[N], s2[N];
#pragma unroll
      for (int k = 0; k < N; ++k) {
        float e = 0.0f, d = 0.0f;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const float cv = row ? c[k + N * j] : c[j + N * k];  // row: k = mx, j = my
          const float t1 = row ? (l ? C.Em[P][j] : C.Em[0][j]) : (l ? C.Dm[P][j] : C.Dm[0][j]);
          const float t2 = row ? (l ? C.Dm[P][j] : C.Dm[0][j]) : (l ? C.Em[P][j] : C.Em[0][j]);
          e = fmaf(t1, cv, e);
          d = fmaf(t2, cv, d);
        }
        s1[k] = e;
        s2[k] = d;
      }
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float bx = 0.0f, by = 0.0f;
#pragma unroll
        for (int k = 0; k < N; ++k) {
          // row: bx[i,l] = sum_mx Dm[i][mx] s1[mx], by[i,l] = sum_mx Em[i][mx] s2[mx]
          // column: bx[l,i] = sum_my Em[i][my] s1[my], by[l,i] = sum_my Dm[i][my] s2[my]
          bx = fmaf(row ? C.Dm[i][k] : C.Em[i][k], s1[k], bx);
          by = fmaf(row ? C.Em[i][k] : C.Dm[i][k], s2[k], by);
        }
        const int lm = row ? i + N * l : l + N * i;
        sbx[lm * NH + h] = hdy * bx;
        sby[lm * NH + h] = hdx * by;
      }
    }
  }
  __syncthreads();
  pdl_launch_dependents();

  // ---- one thread per own cell ------------------------------------------------------------------
  if (NB > NT && threadIdx.x >= NT) return;
  const int tx = threadIdx.x % TX, ty = DIM == 2 ? threadIdx.x / TX : 0;
  const int gi = i0 + tx, gj = j0 + ty;
  if (gi >= nx || gj >= ny) return;
  const int hcx = tx + 1, hcy = DIM == 2 ? ty + 1 : 0;
  const int hc = hcy * HX + hcx;
  const size_t cell = (size_t)gj * nx + gi;
  if (!CVW_SPAN(a.status, cell, 1, a.lim_cell)) return;  // per-cell outputs and rloc
  float c[ND];
#pragma unroll
  for (int m = 0; m < ND; ++m) c[m] = sc[m * NH + hc];
  float n0;
  float wstar[DgTables<DIM, P>::NS];  // unused: CG has no limiter mode
  const float gam = cell_sensor<DIM, P, TX, TY>(a, T, st, sA, c, tx, ty, n0, wstar);
  const Law law(a, c[0]);

  // lambda_e over the volume and face Gauss nodes of the cell polynomial
  float lam = a.lambda_const;
  if (!(a.lambda_const > 0.0f)) {
    lam = 0.0f;
    float tr[4][N];  // right, left, top, bottom traces (tangential modes)
#pragma unroll
    for (int j = 0; j < N; ++j) {
      float r = 0.0f, l = 0.0f, t = 0.0f, b = 0.0f;
      if constexpr (DIM == 1) {
        if (j == 0)
#pragma unroll
          for (int i = 0; i < N; ++i) {
            r += c[i];
            l += (i & 1) ? -c[i] : c[i];
          }
      } else {
#pragma unroll
        for (int i = 0; i < N; ++i) {
          r += c[i + N * j];
          l += (i & 1) ? -c[i + N * j] : c[i + N * j];
          t += c[j + N * i];
          b += (i & 1) ? -c[j + N * i] : c[j + N * i];
        }
      }
      tr[0][j] = r;
      tr[1][j] = l;
      tr[2][j] = t;
      tr[3][j] = b;
    }
#pragma unroll
    for (int q = 0; q < (DIM == 2 ? N : 1); ++q) {
#pragma unroll
      for (int f = 0; f < (DIM == 2 ? 4 : 2); ++f) {
        float v = tr[f][0];
        if constexpr (DIM == 2) {
          v = 0.0f;
#pragma unroll
          for (int j = 0; j < N; ++j) v = fmaf(T.B[q][j], tr[f][j], v);
        }
      lam = fmaxf(lam, law.speed(v));
      }
    }
    // volume nodes, by sum factorisation
#pragma unroll 1
    for (int qx = 0; qx < N; ++qx) {
      float tb[NY1];
#pragma unroll
      for (int my = 0; my < NY1; ++my) {
        float s0 = 0.0f;
#pragma unroll
        for (int mx = 0; mx < N; ++mx) s0 = fmaf(sB[qx * N + mx], c[mx + N * my], s0);
        tb[my] = s0;
      }
#pragma unroll
      for (int qy = 0; qy < NY1; ++qy) {
        float u = tb[0];
        if constexpr (DIM == 2) {
          u = 0.0f;
#pragma unroll
          for (int my = 0; my < N; ++my) u = fmaf(sB[qy * N + my], tb[my], u);
        }
        lam = fmaxf(lam, law.speed(u));
      }
    }
  }
  const float nu = lam * a.nu_scale;
  if (a.gamma_out) a.gamma_out[cell] = gam;
  if (a.nu_out) a.nu_out[cell] = nu;
  if (a.lambda_out) a.lambda_out[cell] = lam;
  if (a.mode & kModeSensorOnly) return;

  // P_h grad u at the own cell's nodes: sum over the cells sharing each node / ML
  float phx[ND], phy[ND];
#pragma unroll
  for (int bb = 0; bb < NY1; ++bb)
#pragma unroll
    for (int aa = 0; aa < N; ++aa) {
      float sx = 0.0f, sy = 0.0f;
      // x-neighbours of the node: (halo column, local index)
      const int ncx = (aa == 0 || aa == P) ? 2 : 1;
      const int ncy = DIM == 2 ? ((bb == 0 || bb == P) ? 2 : 1) : 1;
#pragma unroll
      for (int jy = 0; jy < ncy; ++jy)
#pragma unroll
        for (int jx = 0; jx < ncx; ++jx) {
          int cx = hcx, la = aa, cy = hcy, lb = bb;
          if (aa == 0) { cx = jx == 0 ? hcx - 1 : hcx; la = jx == 0 ? P : 0; }
          if (aa == P) { cx = jx == 0 ? hcx : hcx + 1; la = jx == 0 ? P : 0; }
          if (DIM == 2 && bb == 0) { cy = jy == 0 ? hcy - 1 : hcy; lb = jy == 0 ? P : 0; }
          if (DIM == 2 && bb == P) { cy = jy == 0 ? hcy : hcy + 1; lb = jy == 0 ? P : 0; }
          const int hh = cy * HX + cx, lm = la + N * lb;
          sx += sbx[lm * NH + hh];
          sy += sby[lm * NH + hh];
        }
      // 1 / ML of the node: the inverse lumped masses of its two 1D indices
      const float iml = C.iml[aa == P ? 0 : aa] * a.two_dx * (DIM == 2 ? C.iml[bb == P ? 0 : bb] * a.two_dy : 1.0f);
      phx[aa + N * bb] = sx * iml;
      phy[aa + N * bb] = sy * iml;
    }

  // (d) SC weights (A24) and (e) local residual over the volume Gauss nodes, by sum
  // factorisation: per row qx the x-contractions of c (values, x-derivatives) and of the
  // nodal P_h grad u, then the nodes of the row; the residual is projected back the same way
  bool troubled = a.sc && gam < a.c_gamma && n0 > 1e-30f;
  if (a.troubled_override) {
    const int ov = a.troubled_override[cell];
    if (ov >= 0) troubled = ov && n0 > 1e-30f;
  }
  float afac = -1.0f;
  const bool need_sc = troubled && gam < 1.0f;
  // x-contractions of row qx: tb = B c, td = Bd c (modes), tpx/tpy = Lq ph (nodal)
  auto row = [&](int qx, float (&tb)[NY1], float (&td)[NY1], float (&tpx)[NY1], float (&tpy)[NY1]) {
#pragma unroll
    for (int my = 0; my < NY1; ++my) {
      float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
#pragma unroll
      for (int mx = 0; mx < N; ++mx) {
        const float cm = c[mx + N * my];
        s0 = fmaf(sB[qx * N + mx], cm, s0);
        s1 = fmaf(sBd[qx * N + mx], cm, s1);
        const float lx = (&C.Lq[0][0])[qx * N + mx];
        s2 = fmaf(lx, phx[mx + N * my], s2);
        s3 = fmaf(lx, phy[mx + N * my], s3);
      }
      tb[my] = s0;
      td[my] = s1;
      tpx[my] = s2;
      tpy[my] = s3;
    }
  };
  // node (qx, qy) of the row: value, physical gradient, P_h grad u
  auto node = [&](int qy, const float (&tb)[NY1], const float (&td)[NY1], const float (&tpx)[NY1],
                  const float (&tpy)[NY1], float& u, float& gx, float& gy, float& px, float& py) {
    if constexpr (DIM == 1) {
      u = tb[0];
      gx = td[0] * a.two_dx;
      gy = 0.0f;
      px = tpx[0];
      py = 0.0f;
    } else {
      u = gx = gy = px = py = 0.0f;
#pragma unroll
      for (int my = 0; my < N; ++my) {
        const float by = sB[qy * N + my], ly = (&C.Lq[0][0])[qy * N + my];
        u = fmaf(by, tb[my], u);
        gx = fmaf(by, td[my], gx);
        gy = fmaf(sBd[qy * N + my], tb[my], gy);
        px = fmaf(ly, tpx[my], px);
        py = fmaf(ly, tpy[my], py);
      }
      gx *= a.two_dx;
      gy *= a.two_dy;
    }
  };
  if (need_sc) {
    float s1 = 0.0f, s2 = 0.0f;
#pragma unroll 1
    for (int qx = 0; qx < N; ++qx) {
      float tb[NY1], td[NY1], tpx[NY1], tpy[NY1];
      row(qx, tb, td, tpx, tpy);
      float X[N][NY1];  // X[kx][my] = sum_mx Bk[kx][qx][mx] c[mx, my]
#pragma unroll
      for (int kx = 0; kx < N; ++kx)
#pragma unroll
        for (int my = 0; my < NY1; ++my) {
          float acc = 0.0f;
#pragma unroll
          for (int mx = 0; mx < N; ++mx) acc = fmaf(sBk[(kx * N + qx) * N + mx], c[mx + N * my], acc);
          X[kx][my] = acc;
        }
#pragma unroll 1
      for (int qy = 0; qy < NY1; ++qy) {
        float u, gx, gy, px, py;
        node(qy, tb, td, tpx, tpy, u, gx, gy, px, py);
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
        const int q = qx + N * qy;
        sNq[q * NT + threadIdx.x] = nq;
        const float f = fmaf(gx, gx, gy * gy) - gam * (gx * px + gy * py);
        const float W = sW[qx] * (DIM == 2 ? sW[qy] : 1.0f);
        s1 = fmaf(W, f, s1);
        s2 = fmaf(W * nq, f, s2);
      }
    }
    if (s1 > 0.0f && s2 > 0.0f) afac = s1 / s2;
  }
  if (a.troubled_out) a.troubled_out[cell] = troubled ? 1 : 0;
  if (a.alpha_out) {
#pragma unroll 1
    for (int q = 0; q < ND; ++q) a.alpha_out[cell * ND + q] = afac >= 0.0f ? sNq[q * NT + threadIdx.x] * afac : 1.0f;
  }
  float r[ND];
#pragma unroll
  for (int m = 0; m < ND; ++m) r[m] = 0.0f;
#pragma unroll 1
  for (int qx = 0; qx < N; ++qx) {
    float tb[NY1], td[NY1], tpx[NY1], tpy[NY1];
    row(qx, tb, td, tpx, tpy);
    float hx[NY1], hy[NY1];
#pragma unroll
    for (int b = 0; b < NY1; ++b) hx[b] = hy[b] = 0.0f;
#pragma unroll 1
    for (int qy = 0; qy < NY1; ++qy) {
      float u, gx, gy, px, py;
      node(qy, tb, td, tpx, tpy, u, gx, gy, px, py);
      // f(u) - f(ubar): the cell constant f(ubar) contributes f(ubar) int_K grad phi_a,
      // which lives on the cell's edges and telescopes between neighbours (added below)
      float fx, fy;
      law.flux_dev(u - c[0], fx, fy);
      const int q = qx + N * qy;
      const float al = afac >= 0.0f ? sNq[q * NT + threadIdx.x] * afac : 1.0f;
      const float W = sW[qx] * (DIM == 2 ? sW[qy] : 1.0f) * hdx * hdy;
      const float Gx = W * (fx - nu * al * (gx - gam * px));
      const float Gy = W * (fy - nu * al * (gy - gam * py));
      if constexpr (DIM == 2) {
#pragma unroll
        for (int b = 0; b < N; ++b) {
          hx[b] = fmaf((&C.Lq[0][0])[qy * N + b], Gx, hx[b]);
          hy[b] = fmaf((&C.Ldq[0][0])[qy * N + b], Gy, hy[b]);
        }
      } else {
        hx[0] += Gx;
      }
    }
    // r[a, b] += 2/dx Ldq[qx][a] hx[b] + 2/dy Lq[qx][a] hy[b]
#pragma unroll
    for (int b = 0; b < NY1; ++b)
#pragma unroll
      for (int aa = 0; aa < N; ++aa) {
        float v = fmaf(a.two_dx * (&C.Ldq[0][0])[qx * N + aa], hx[b], r[aa + N * b]);
        if constexpr (DIM == 2) v = fmaf(a.two_dy * (&C.Lq[0][0])[qx * N + aa], hy[b], v);
        r[aa + N * b] = v;
      }
  }
  // The constant part of the flux: int_K d_x phi_ab f(ubar_e) = (delta_{a,p} - delta_{a,0})
  // wl_b (dy/2) f_x(ubar_e) (likewise in y).  At the nodes of an edge between a left cell L
  // and a right cell R the two cells' terms sum to (f_x(ubar_L) - f_x(ubar_R)) wl_b dy/2;
  // each cell adds that sum for its left and bottom edges (its right and top edges are
  // its neighbours' left and bottom ones), the difference formed by the deviation formula
  // of its own law from the halo means.
  {
    float fx, fy;
    law.flux_dev(sc[hc - 1] - c[0], fx, fy);  // f(ubar_left) - f(ubar_e)
#pragma unroll
    for (int b = 0; b < NY1; ++b) r[N * b] = fmaf(fx, DIM == 2 ? C.wl[b] * hdy : 1.0f, r[N * b]);
    if constexpr (DIM == 2) {
      law.flux_dev(sc[hc - HX] - c[0], fx, fy);  // f(ubar_below) - f(ubar_e)
#pragma unroll
      for (int aa = 0; aa < N; ++aa) r[aa] = fmaf(fy, C.wl[aa] * hdx, r[aa]);
    }
  }
  if constexpr (ND % 4 == 0) {  // rloc is mesh-owned (aligned): 16-byte stores
#pragma unroll
    for (int q = 0; q < ND / 4; ++q)
      reinterpret_cast<float4*>(a.rloc + cell * ND)[q] = make_float4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
  } else {
#pragma unroll
    for (int m = 0; m < ND; ++m) a.rloc[cell * ND + m] = r[m];
  }
}

// Nodal assembly r_j at lattice node (I, J), 0 <= I < nnx, 0 <= J < nny: the sum of the
// cell-local residuals (which carry the telescoped flux of the cell means) over the
// cells containing the node, in a fixed order: the cell below-left of the node first,
// then the one to its right, then the row above.  A node with local index a = 0 in x
// lies in cell i - 1 (as its local p) and cell i (as its local 0); likewise in y.
template <int DIM, int P>
__device__ __forceinline__ float node_residual(const StageArgs& a, int I, int J) {
  constexpr int N = P + 1, ND = DIM == 2 ? N * N : N;
  const int nx = a.nx;
  const int i = I / P, aa = I - i * P;
  const int cx0 = aa == 0 ? (i == 0 ? nx - 1 : i - 1) : i, lx0 = aa == 0 ? P : aa;
  const int64_t lim = CVW_EXTENT(a, lim_cell) * ND;
  auto rl = [&](size_t k) { return CVW_SPAN(a.status, k, 1, lim) ? a.rloc[k] : 0.0f; };
  if constexpr (DIM == 1) {
    float r = rl((size_t)cx0 * ND + lx0);
    if (aa == 0) r += rl((size_t)i * ND);
    return r;
  } else {
    const int j = J / P, bb = J - j * P;
    const int cy0 = bb == 0 ? (j == 0 ? a.ny - 1 : j - 1) : j, ly0 = bb == 0 ? P : bb;
    const size_t row0 = (size_t)cy0 * nx, row1 = (size_t)j * nx;
    float r = rl((row0 + cx0) * ND + lx0 + N * ly0);
    if (aa == 0) r += rl((row0 + i) * ND + N * ly0);
    if (bb == 0) {
      r += rl((row1 + cx0) * ND + lx0);
      if (aa == 0) r += rl((row1 + i) * ND);
    }
    return r;
  }
}

// 1D nodal assembly: r_j and du = r_j / ML_j.
template <int DIM, int P>
__global__ void cg_node_rhs(const __grid_constant__ StageArgs a, const __grid_constant__ CgTables<DIM, P> C) {
  const int64_t nn = (int64_t)a.nnx * (DIM == 2 ? a.nny : 1);
  const float hdx = 1.0f / a.two_dx, hdy = DIM == 2 ? 1.0f / a.two_dy : 1.0f;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nn; j += (int64_t)gridDim.x * blockDim.x) {
    const int I = (int)(j % a.nnx), J = (int)(j / a.nnx);
    const float r = node_residual<DIM, P>(a, I, J);
    const float ml = ml1(C, I % P, hdx) * (DIM == 2 ? ml1(C, J % P, hdy) : 1.0f);
    if (!CVW_SPAN(a.status, j, 1, a.lim_out)) continue;
    a.rnode[j] = r;
    a.du[j] = r / ml;
  }
}

// (M_C du) at lattice node (I, J): the consistent mass is the tensor product of the 1D
// assembled masses, so the product is a sum over the (up to two) cells containing the
// node in each direction of M1[local][b] times the nodes of that cell, x first, then y.
template <int DIM, int P>
__device__ __forceinline__ float mass_apply(const CgTables<DIM, P>& C, const float* __restrict__ du, int I, int J,
                                            int nnx, int nny, float hdx, float hdy) {
  const int ax = I % P, ay = DIM == 2 ? J % P : 0;
  const int ncx = ax == 0 ? 2 : 1, ncy = DIM == 2 ? (ay == 0 ? 2 : 1) : 1;
  float acc = 0.0f;
  for (int ky = 0; ky < ncy; ++ky) {
    // y-cell starting at lattice row J0y, node's local index ly in it
    const int ly = DIM == 2 ? (ay == 0 ? (ky == 0 ? P : 0) : ay) : 0;
    const int J0y = J - ly;
#pragma unroll
    for (int d = 0; d < (DIM == 2 ? P + 1 : 1); ++d) {
      const int Jr = DIM == 2 ? ((J0y + d) % nny + nny) % nny : 0;
      const float* rowp = du + (size_t)Jr * nnx;
      float w = 0.0f;
      for (int kx = 0; kx < ncx; ++kx) {
        const int lx = ax == 0 ? (kx == 0 ? P : 0) : ax;
        const int I0x = I - lx;
#pragma unroll
        for (int b = 0; b <= P; ++b) w = fmaf(C.M1[lx][b], rowp[((I0x + b) % nnx + nnx) % nnx], w);
      }
      acc = DIM == 2 ? fmaf(C.M1[ly][d], w, acc) : w;
    }
  }
  return acc * hdx * hdy;
}

// One defect-correction sweep du_out = du_in + ML^{-1}(r - M_C du_in) (reading A12), node
// by node (1D meshes); the final sweep writes the SSP-RK3 combination (or du itself).
template <int DIM, int P>
__global__ void cg_node_sweep(const __grid_constant__ StageArgs a, const __grid_constant__ CgTables<DIM, P> C,
                              const float* __restrict__ du_in, float* __restrict__ du_out, int final_sweep) {
  const int64_t nn = (int64_t)a.nnx * (DIM == 2 ? a.nny : 1);
  const float hdx = 1.0f / a.two_dx, hdy = DIM == 2 ? 1.0f / a.two_dy : 1.0f;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nn; j += (int64_t)gridDim.x * blockDim.x) {
    if (!CVW_SPAN(a.status, j, 1, a.lim_out)) continue;  // nodal inputs, outputs and work arrays
    const int I = (int)(j % a.nnx), J = (int)(j / a.nnx);
    const float mc = mass_apply<DIM, P>(C, du_in, I, J, a.nnx, DIM == 2 ? a.nny : 1, hdx, hdy);
    const float ml = ml1(C, I % P, hdx) * (DIM == 2 ? ml1(C, J % P, hdy) : 1.0f);
    const float du = du_in[j] + (a.rnode[j] - mc) / ml;
    if (!final_sweep) {
      du_out[j] = du;
    } else if (a.mode & kModeRK) {
      float v = fmaf(a.dt, du, a.u_in[j]);
      if (a.rk_a != 0.0f) v = fmaf(a.rk_b, v - a.u_n[j], a.u_n[j]);  // plain load: u_n may alias u_out
      a.u_out[j] = v;
      if (!isfinite(v)) atomicOr(a.status, kStatNonfinite);
    } else {
      a.u_out[j] = du;
      if (!isfinite(du)) atomicOr(a.status, kStatNonfinite);
    }
  }
}

// The node phase of one 2D stage, per tile of kNdX x kNdY lattice nodes: the nodal
// assembly r and du0 = r / ML on the tile and a halo of 2p nodes, the first
// defect-correction sweep du1 = du0 + ML^{-1}(r - M_C du0) (reading A12) on the tile and a
// halo of p nodes, and the second at the tile's nodes, which writes the SSP-RK3
// combination (or du itself for a residual).  The consistent mass is the tensor product
// of the 1D assembled masses, so M_C du is applied as two passes over the window: along
// x (each node sums M1[local][b] du over the nodes of the up to two cells containing it),
// then along y.  The halo values are recomputed by every tile that needs them, in the same
// arithmetic, so neighbouring tiles agree bitwise.
// 32x32 tiles of 1024 threads from p = 3 on, 32x16 of 512 threads below (measured)
constexpr int kNdX = 32;
template <int P>
__host__ __device__ constexpr int node_tile_y() { return P >= 3 ? 32 : 16; }


template <int P>
__global__ void __launch_bounds__(kNdX* node_tile_y<P>(), 2048 / (kNdX * node_tile_y<P>()))
    cg_node_stage2d(const __grid_constant__ StageArgs a, const __grid_constant__ CgTables<2, P> C) {
  constexpr int kNdY = node_tile_y<P>();
  constexpr int N = P + 1, NT = kNdX * kNdY;
  constexpr int RX = kNdX + 4 * P, RY = kNdY + 4 * P;  // r and du0 window (halo 2p)
  constexpr int DX = kNdX + 2 * P, DY = kNdY + 2 * P;  // du1 window (halo p)
  __shared__ float sr[RY][RX];
  __shared__ float sd0[RY][RX];
  __shared__ float sxp[RY * DX];  // x-pass of M_C du0 [RY][DX], then of M_C du1 [DY][kNdX]
  __shared__ float sd1[DY][DX];
  __shared__ float sM1[N][N];
  // per window column rx (lattice column I0 - 2p + rx) and row ry: the offsets of the
  // local residual entries the node gathers (B: the second cell, -1 if none), the node's
  // 1D local index and its inverse 1D lumped mass
  __shared__ long long srowA[RY], srowB[RY];
  __shared__ int scolA[RX], scolB[RX], slx[RX], sly[RY];
  __shared__ float simlx[RX], simly[RY];
  const int nnx = a.nnx, nny = a.nny;
  const int I0 = blockIdx.x * kNdX, J0 = blockIdx.y * kNdY;
  const float hh = (1.0f / a.two_dx) * (1.0f / a.two_dy), k2 = a.two_dx * a.two_dy;
  if (threadIdx.x < N * N) sM1[threadIdx.x / N][threadIdx.x % N] = (&C.M1[0][0])[threadIdx.x];
  // this thread's output node; its RK inputs are loaded right after pdl_wait, so that their
  // latency overlaps the window (u_n may alias u_out: only this thread reads or writes
  // node j)
  const int tx = threadIdx.x % kNdX, ty = threadIdx.x / kNdX;
  const int I = I0 + tx, J = J0 + ty;
  const bool own = I < nnx && J < nny;
  const size_t j = own ? (size_t)J * nnx + I : 0;
  const bool rk = (a.mode & kModeRK) != 0, with_un = rk && a.rk_a != 0.0f;
  float uin = 0.0f, un = 0.0f;
  // 1 / (m_l wl[l]) of 1D local index l in [0, p)
  auto iml = [&](int l) {
    float v = C.iml[0];
#pragma unroll
    for (int k = 1; k < P; ++k) v = l == k ? C.iml[k] : v;
    return v;
  };
  // A node with 1D local index 0 lies in two cells (the one before it as its local p),
  // any other in one; the nodal sum takes the cells below-left first (node_residual's order).
  if (threadIdx.x < RX) {
    const int rx = threadIdx.x, Iw = wrap_index(I0 - 2 * P + rx, nnx), i = Iw / P, aa = Iw - i * P;
    const int cx0 = aa == 0 ? (i == 0 ? a.nx - 1 : i - 1) : i;
    scolA[rx] = cx0 * (N * N) + (aa == 0 ? P : aa);
    scolB[rx] = aa == 0 ? i * (N * N) : -1;
    slx[rx] = aa;
    simlx[rx] = iml(aa);
  } else if (threadIdx.x < RX + RY) {
    const int ry = threadIdx.x - RX, Jw = wrap_index(J0 - 2 * P + ry, nny), jc = Jw / P, bb = Jw - jc * P;
    const int cy0 = bb == 0 ? (jc == 0 ? a.ny - 1 : jc - 1) : jc;
    const long long rowlen = (long long)a.nx * (N * N);
    srowA[ry] = cy0 * rowlen + N * (bb == 0 ? P : bb);
    srowB[ry] = bb == 0 ? jc * rowlen : -1;
    sly[ry] = bb;
    simly[ry] = iml(bb);
  }
  pdl_wait();  // everything below reads or writes what earlier kernels write
  const bool own_ok = own && CVW_SPAN(a.status, j, 1, a.lim_in) && CVW_SPAN(a.status, j, 1, a.lim_out);
  if (own_ok && rk) uin = a.u_in[j];
  if (own_ok && with_un) un = a.u_n[j];
  __syncthreads();
  // ---- r and du0 on the window: every gather of the thread in flight before the first use -----
  constexpr int NW = (RX * RY + NT - 1) / NT;
  float rv[NW];
#pragma unroll
  for (int k = 0; k < NW; ++k) {
    const int f = threadIdx.x + k * NT;
    rv[k] = 0.0f;
    if (f < RX * RY) {
      const int ry = f / RX, rx = f - ry * RX;
      const long long rA = srowA[ry], rB = srowB[ry];
      const int cA = scolA[rx], cB = scolB[rx];
      const int64_t lim = CVW_EXTENT(a, lim_cell) * (N * N);
      auto rl = [&](long long k) { return CVW_SPAN(a.status, k, 1, lim) ? a.rloc[k] : 0.0f; };
      float r = rl(rA + cA);
      if (cB >= 0) r += rl(rA + cB);
      if (rB >= 0) {
        r += rl(rB + cA);
        if (cB >= 0) r += rl(rB + cB);
      }
      rv[k] = r;
    }
  }
#pragma unroll
  for (int k = 0; k < NW; ++k) {
    const int f = threadIdx.x + k * NT;
    if (f < RX * RY) {
      const int ry = f / RX, rx = f - ry * RX;
      sr[ry][rx] = rv[k];
      sd0[ry][rx] = rv[k] * (simlx[rx] * simly[ry] * k2);
    }
  }
  __syncthreads();
  // The passes work cell by cell: a cell's p+1 nodes along the pass direction (and the p
  // nodes of the cell before it, for the node shared by both) are read once, and its p
  // outputs follow with compile-time local indices: output a of the cell sums
  // M1[a][b] over the cell's nodes, plus M1[p][b] over the previous cell's for a = 0.
  // Segment s of a line starts at the cell whose local node 0 sits at source index
  // z = out0 - a0 + s p (a0: the local index of the line's first output); the products
  // are taken in the same order as node by node, so the results are the same bits.
  auto cell_pass = [&](const float (&v)[2 * P + 1], int a) {
    float w = 0.0f;
    if (a == 0) {
#pragma unroll
      for (int b = 0; b <= P; ++b) w = fmaf(C.M1[P][b], v[b], w);
#pragma unroll
      for (int b = 0; b <= P; ++b) w = fmaf(C.M1[0][b], v[P + b], w);
    } else {
#pragma unroll
      for (int aa = 1; aa < P; ++aa)
        if (aa == a) {
#pragma unroll
          for (int b = 0; b <= P; ++b) w = fmaf(C.M1[aa][b], v[P + b], w);
        }
    }
    return w;
  };
  // ---- first sweep: x-pass over the rows of the window, columns of the du1 window ----------
  {
    constexpr int NSEG = (DX + P - 1) / P + 1;
    const int a0 = slx[P];
    for (int f = threadIdx.x; f < RY * NSEG; f += NT) {
      const int ry = f / NSEG, sg = f - ry * NSEG, z = P - a0 + sg * P;  // r-window column of node 0
      float v[2 * P + 1];
#pragma unroll
      for (int j = 0; j <= 2 * P; ++j) {
        const int col = z - P + j;
        v[j] = col >= 0 && col < RX ? sd0[ry][col] : 0.0f;
      }
#pragma unroll
      for (int a = 0; a < P; ++a) {
        const int cx = z - P + a;  // du1-window column
        if (cx >= 0 && cx < DX) sxp[ry * DX + cx] = cell_pass(v, a);
      }
    }
  }
  __syncthreads();
  // ---- first sweep: y-pass and du1 -----------------------------------------------------------
  {
    constexpr int NSEG = (DY + P - 1) / P + 1;
    const int b0 = sly[P];
    for (int f = threadIdx.x; f < DX * NSEG; f += NT) {
      const int cx = f / NSEG, sg = f - cx * NSEG, z = P - b0 + sg * P;  // r-window row of node 0
      const int rx = cx + P;
      float v[2 * P + 1];
#pragma unroll
      for (int j = 0; j <= 2 * P; ++j) {
        const int row = z - P + j;
        v[j] = row >= 0 && row < RY ? sxp[row * DX + cx] : 0.0f;
      }
#pragma unroll
      for (int a = 0; a < P; ++a) {
        const int dy = z - P + a, ry = dy + P;
        if (dy >= 0 && dy < DY) {
          const float mc = cell_pass(v, a);
          sd1[dy][cx] = sd0[ry][rx] + (sr[ry][rx] - mc * hh) * (simlx[rx] * simly[ry] * k2);
        }
      }
    }
  }
  __syncthreads();
  // ---- second sweep: x-pass over the du1 window's rows, the tile's columns ------------------
  {
    constexpr int NSEG = (kNdX + P - 1) / P + 1;
    const int a0 = slx[2 * P];
    for (int f = threadIdx.x; f < DY * NSEG; f += NT) {
      const int dy = f / NSEG, sg = f - dy * NSEG, z = P - a0 + sg * P;  // du1-window column of node 0
      float v[2 * P + 1];
#pragma unroll
      for (int j = 0; j <= 2 * P; ++j) {
        const int col = z - P + j;
        v[j] = col >= 0 && col < DX ? sd1[dy][col] : 0.0f;
      }
#pragma unroll
      for (int a = 0; a < P; ++a) {
        const int ox = z - P + a;
        if (ox >= 0 && ox < kNdX) sxp[dy * kNdX + ox] = cell_pass(v, a);
      }
    }
  }
  __syncthreads();
  pdl_launch_dependents();
  if (!own_ok) return;
  // ---- second sweep: y-pass at this thread's node, and the stage output ----------------------
  const int ay = sly[ty + 2 * P], ly0 = ay == 0 ? P : ay, dy = ty + P;
  float mc = 0.0f;
#pragma unroll
  for (int d = 0; d <= P; ++d) mc = fmaf(sM1[ly0][d], sxp[(dy - ly0 + d) * kNdX + tx], mc);
  if (ay == 0) {
#pragma unroll
    for (int d = 0; d <= P; ++d) mc = fmaf(sM1[0][d], sxp[(dy + d) * kNdX + tx], mc);
  }
  const float du = sd1[dy][tx + P] + (sr[ty + 2 * P][tx + 2 * P] - mc * hh) * (simlx[tx + 2 * P] * simly[ty + 2 * P] * k2);
  if (rk) {
    float v = fmaf(a.dt, du, uin);
    if (with_un) v = fmaf(a.rk_b, v - un, un);
    a.u_out[j] = v;
    if (!isfinite(v)) atomicOr(a.status, kStatNonfinite);
  } else {
    a.u_out[j] = du;
    if (!isfinite(du)) atomicOr(a.status, kStatNonfinite);
  }
}

template <int DIM, int P, int SYS, int TX, int TY>
cudaError_t launch_cg_t(const cvweno_mesh_s* m, const StageArgs& a, cudaStream_t s) {
  using Tb = DgTables<DIM, P>;
  using Cb = CgTables<DIM, P>;
  constexpr size_t smem = CgLayout<DIM, P, TX, TY>::BYTES;
  static_assert(smem <= 220 * 1024, "tile too large for shared memory");
  if (m->tables_bytes != sizeof(Tb) || m->cg_tables_bytes != sizeof(Cb)) return cudaErrorInvalidValue;
  const Tb& T = *static_cast<const Tb*>(m->tables);
  const Cb& C = *static_cast<const Cb*>(m->cg_tables);
  auto k1 = cg_stage_cells<DIM, P, SYS, TX, TY>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((a.nx + TX - 1) / TX, DIM == 2 ? (a.ny + TY - 1) / TY : 1);
  cudaError_t e = launch_pdl(k1, grid, dim3(cg_block_threads<DIM, P, TX, TY>()), smem, s, a, T, C);
  if (e != cudaSuccess) return e;
  if (a.mode & kModeSensorOnly) return cudaGetLastError();
  kernel_mark(m, s);
  if constexpr (DIM == 2) {
    constexpr int kNdY = node_tile_y<P>();
    const dim3 ng((a.nnx + kNdX - 1) / kNdX, (a.nny + kNdY - 1) / kNdY);
    e = launch_pdl(cg_node_stage2d<P>, ng, dim3(kNdX * kNdY), 0, s, a, C);
    if (e != cudaSuccess) return e;
    kernel_mark(m, s);
  } else {
    const int64_t nn = m->nnode;
    const int bn = (int)((nn + 255) / 256 < 4096 ? (nn + 255) / 256 : 4096);
    cg_node_rhs<DIM, P><<<bn, 256, 0, s>>>(a, C);
    kernel_mark(m, s);
    cg_node_sweep<DIM, P><<<bn, 256, 0, s>>>(a, C, a.du, a.du2, 0);
    kernel_mark(m, s);
    cg_node_sweep<DIM, P><<<bn, 256, 0, s>>>(a, C, a.du2, nullptr, 1);
    kernel_mark(m, s);
  }
  return cudaGetLastError();
}

template <int DIM, int P>
cudaError_t launch_cg_p(const cvweno_mesh_s* m, const StageArgs& a, cudaStream_t s) {
  constexpr int TX = DIM == 2 ? 16 : 128, TY = DIM == 2 ? 8 : 1;
  switch (m->desc.system) {
    case CVWENO_BURGERS: return launch_cg_t<DIM, P, CVWENO_BURGERS, TX, TY>(m, a, s);
    case CVWENO_KPP: return DIM == 2 ? launch_cg_t<DIM, P, CVWENO_KPP, TX, TY>(m, a, s) : cudaErrorNotSupported;
    case CVWENO_LINADV: return launch_cg_t<DIM, P, CVWENO_LINADV, TX, TY>(m, a, s);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace

cudaError_t launch_stage_cg(const cvweno_mesh_s* m, const StageArgs& a, cudaStream_t s) {
  switch (m->dim * 10 + m->p) {
    case 11: return launch_cg_p<1, 1>(m, a, s);
    case 12: return launch_cg_p<1, 2>(m, a, s);
    case 13: return launch_cg_p<1, 3>(m, a, s);
    case 14: return launch_cg_p<1, 4>(m, a, s);
    case 21: return launch_cg_p<2, 1>(m, a, s);
    case 22: return launch_cg_p<2, 2>(m, a, s);
    case 23: return launch_cg_p<2, 3>(m, a, s);
    case 24: return launch_cg_p<2, 4>(m, a, s);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace cvw
