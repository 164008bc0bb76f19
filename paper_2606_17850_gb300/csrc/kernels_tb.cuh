// Temporal blocking of the Chebyshev preconditioner (layer-uniform grids).
//
// The preconditioner's steps need no reductions (Sec. 4.3: only SpMVs and AXPYs),
// so several of them can run inside one kernel on a tile.  For S steps a tile is
// (32 - 2S) x (EY - 2S) columns (all layers) grown by an S-cell halo in x and y.  Each thread owns one
// column of the grown tile and keeps that column's z_m, z_{m-1} and r in registers;
// per step it publishes z_m into a shared-memory plane, reads its four in-plane
// neighbours from there (the z neighbours are its own registers) and forms z_{m+1}.
// The region whose neighbours are still valid shrinks by one cell per step, so
// after the S <= TB_H steps the tile interior holds z_{m+S}.
//
// Blackwell data movement: the kernel is persistent (one CTA per SM walks the tile
// list) and the next tile's three input boxes (z_m, z_{m-1}, r: TB_BW x EY x L
// floats each) are fetched by the tensor memory accelerator into a staging buffer
// while the current tile computes; completion is tracked by an mbarrier.  Two plane
// buffers alternate between steps, so a step needs a single CTA barrier.
//
// Per-layer constants (face conductances of the layer table, the diagonal of an
// interior cell, the inverse diagonal for every in-plane boundary case) and the
// step coefficients are kernel parameters, so the stencil's multiplications take
// them straight from the constant bank.  The product is taken in expanded form,
// (A v)_i = d v_i - gx (v_E + v_W) - gy (v_N + v_S) - gzu v_U - gzd v_D, the
// diagonal-plus-off-diagonals form of the paper's stored product (Algorithm 3),
// with d the diagonal of a cell that has all four in-plane faces.  A missing
// neighbour (domain edge) is read as the cell itself: its -g v_i cancels the g v_i
// that d holds for the absent face, which is the adiabatic boundary.  Seven FP32
// operations per cell instead of the difference form's thirteen; the result equals
// the one-step kernels' difference form up to rounding.  With the Jacobi scaling
// D^-1 r is formed once per tile, so a step's update is one FMA more than the
// stencil: z_{m+1} = z_m + c1 (z_m - z_{m-1}) + c2 (D^-1 r - D^-1 A z_m).
//
// DRAM traffic per S steps: the three inputs once plus one or two outputs
// (about 20 B/cell) instead of 16 B/cell per step.
#pragma once

#include <cuda.h>

#include "common.cuh"

#define TB_H 4    // most steps per launch
#define TB_EX 32  // grown tile width in threads: one warp per row
#define TB_BW 36  // staged box width: the grown tile's first column rounded down to 16 bytes, + 32
// bounded mbarrier wait: give up after about one second of device time
#define TB_WAIT_NS 1000000000ull
// test hook: limit of the wait on a barrier phase that nothing completes
#define TB_TEST_WAIT_NS 2000000ull

// The step works on layer pairs (k, k + LMAX/2): the per-layer constants of a pair
// sit side by side, as the operands of Blackwell's paired FP32 instructions, so a
// pair's vertical neighbours are the pairs k + 1 and k - 1 (except across the
// middle of the column, one scalar term at each end); the faces are stored negated
// (d v - gx (v_E + v_W) - ... becomes fused multiply-adds without a negation).
template <int LMAX>
struct __align__(8) TBParams {
  float2 c1[TB_H], c2[TB_H];    // Chebyshev step coefficients of this chunk, (c, c)
  float2 d[LMAX / 2];           // diagonal of a cell with all four in-plane faces
  float2 ngx[LMAX / 2], ngy[LMAX / 2];  // -(in-plane face conductances)
  float2 ngzu[LMAX / 2], ngzd[LMAX / 2];  // -(face to the layer above / below), 0 at the ends
  float invd[9][LMAX];          // 1 / diagonal for (x faces present) + 3 (y faces present)
  float z1s;                    // first chunk: z_1 = z1s D^-1 r, formed from the staged r
  int expire_test;              // test hook: the first wait of each CTA runs out (see below)
};

__device__ __forceinline__ unsigned tb_smem(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tb_mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tb_smem(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void tb_mbar_expect(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tb_smem(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool tb_mbar_try(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(tb_smem(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long tb_clock_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// true when the phase completed; false after about limit_ns of device time
__device__ __forceinline__ bool tb_mbar_wait(unsigned long long* bar, unsigned parity,
                                             unsigned long long limit_ns = TB_WAIT_NS) {
  if (tb_mbar_try(bar, parity)) return true;
  const unsigned long long t0 = tb_clock_ns();
  while (!tb_mbar_try(bar, parity))
    if (tb_clock_ns() - t0 > limit_ns) return false;
  return true;
}

__device__ __forceinline__ void tb_tma_3d(float* dst, const CUtensorMap* map, int x, int y, int z,
                                          unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(tb_smem(dst)),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(tb_smem(bar))
      : "memory");
}

// dynamic shared memory of one CTA: staging (3 boxes) + two planes + two mbarriers
// (the staged loads' and the test hook's), plus room to align the staging boxes to
// 128 bytes
template <int LMAX, int EY>
constexpr size_t tb_smem_bytes() {
  return ((size_t)3 * LMAX * EY * TB_BW + (size_t)2 * LMAX * EY * TB_EX) * sizeof(float) + 16 + 128;
}

// STEPS steps with a halo of STEPS cells: the interior is (32 - 2 STEPS) x
// (EY - 2 STEPS) columns.  Layers L..LMAX-1 (when the stack has fewer than LMAX
// layers) are carried as zeros: their coefficients and inverse diagonal are 0, so
// they stay 0 and the step loop needs no per-layer guard.
//
// FIRST: the chunk starts the polynomial: z_1 = z1s D^-1 r and z_0 = 0 are formed from
// the staged r, so only the r box is staged and z_1 is never stored.
template <int LMAX, int EY, int STEPS, bool SCALED, bool LAST, bool FIRST>
__global__ void __launch_bounds__(TB_EX * EY, 1)
    k_cheb_tb(Dims d, int ntx, int ntiles, int has_prev, Ctl* ctl,
              const __grid_constant__ CUtensorMap m_cur, const __grid_constant__ CUtensorMap m_prev,
              const __grid_constant__ CUtensorMap m_r, float* __restrict__ out_cur, float* __restrict__ out_prev,
              const __grid_constant__ TBParams<LMAX> P, double* partials, int stride, unsigned* counter) {
  if (ld_int(&ctl->done)) return;
  constexpr int H = STEPS;
  constexpr int TX = TB_EX - 2 * H, TY = EY - 2 * H;  // interior of a tile
  static_assert(LMAX % 2 == 0, "layers are processed in pairs");
  constexpr int LP = LMAX / 2;  // layer pairs
  constexpr int PL = EY * TB_EX;  // floats per layer plane
  constexpr int SL = EY * TB_BW;  // floats per staged layer
  extern __shared__ __align__(128) float tb_dyn[];
  float* tb_sm = tb_dyn + (((128u - (tb_smem(tb_dyn) & 127u)) & 127u) >> 2);  // 128-byte aligned
  float* stage = tb_sm;                    // [3][LMAX][EY][TB_BW]: z_m, z_{m-1}, r
  float* plane = tb_sm + 3 * LMAX * SL;    // [2][LMAX][EY][TB_EX]
  unsigned long long* bar = (unsigned long long*)(plane + 2 * LMAX * PL);
  const int L = d.L;
  const int ex = threadIdx.x, ey = threadIdx.y;
  const int tid = ex + TB_EX * ey;
  const unsigned box_bytes = (unsigned)(L * SL * sizeof(float));
  const unsigned tx_bytes = box_bytes * (FIRST ? 1u : (has_prev ? 3u : 2u));

  // Layers L..LMAX-1 of the three boxes, and the whole z_{m-1} box when there is
  // none, are never written by the tensor copies: zero them once, so the staged
  // loads below need no per-layer guard.
  for (int b = 0; b < 3; ++b) {
    const int z0 = (b == 1 && !has_prev) ? 0 : L;
    for (int i = tid; i < (LMAX - z0) * SL; i += TB_EX * EY) stage[(b * LMAX + z0) * SL + i] = 0.f;
  }
  if (tid == 0) {
    tb_mbar_init(bar, 1);
    tb_mbar_init(bar + 1, 1);  // test hook only: no thread ever arrives on it
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  // the box starts at the grown tile's first column rounded down to a multiple of 4
  // cells (a 16-byte boundary, as the tensor copy requires)
  auto issue = [&](int tx, int ty) {
    const int xa = (tx * TX - H) & ~3, y0 = ty * TY - H;
    tb_mbar_expect(bar, tx_bytes);
    if (!FIRST) tb_tma_3d(stage, &m_cur, xa, y0, 0, bar);
    if (has_prev && !FIRST) tb_tma_3d(stage + LMAX * SL, &m_prev, xa, y0, 0, bar);
    tb_tma_3d(stage + 2 * LMAX * SL, &m_r, xa, y0, 0, bar);
  };
  // tile t = tx + ntx ty, advanced by gridDim.x without a division per tile
  const int dtx = (int)gridDim.x % ntx, dty = (int)gridDim.x / ntx;
  auto advance = [&](int& tx, int& ty) {
    tx += dtx;
    ty += dty;
    if (tx >= ntx) {
      tx -= ntx;
      ++ty;
    }
  };
  int tx = (int)blockIdx.x % ntx, ty = (int)blockIdx.x / ntx;
  if (tid == 0 && (int)blockIdx.x < ntiles) issue(tx, ty);

  float part[1] = {0.f};
  unsigned parity = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    // With the test hook the CTA first waits on a phase of the second barrier that
    // nothing completes, so that wait runs out after TB_TEST_WAIT_NS and the expiry
    // path below runs with this tile's copy still outstanding or just landed.
    bool ok = !(P.expire_test && t == (int)blockIdx.x) || tb_mbar_wait(bar + 1, 0u, TB_TEST_WAIT_NS);
    if (ok) ok = tb_mbar_wait(bar, parity);
    if (__syncthreads_or(!ok)) {
      // Expiry: record the error and end the solve's loops, then wait (bounded
      // again) for this tile's tensor copy, so the CTA never exits while a copy
      // into its shared memory may still be in flight.  No later copy was issued.
      if (tid == 0) {
        tb_mbar_wait(bar, parity);
        atomicCAS(&ctl->status, 0, 3);  // TH_ECUDA, unless an error is recorded already
        ctl->outer_done = 1;
        __threadfence();
        atomicExch(&ctl->done, 1);
      }
      break;
    }
    parity ^= 1u;
    const int x0 = tx * TX - H;
    const int gx = x0 + ex;
    const int gy = ty * TY - H + ey;
    const int st = ey * TB_BW + ex + (x0 - (x0 & ~3));  // this column in a staged layer
    const bool inside = gx >= 0 && gx < d.nx && gy >= 0 && gy < d.ny;
    // za / zb hold z_m / z_{m-1} and swap roles every step: a step writes z_{m+1}
    // over z_{m-1}, so no register moves are needed.  A row that skips a step keeps
    // stale values in the swapped arrays; it lies outside the valid region from then
    // on and is read only by rows that are outside it too.
    // Registers hold layer pairs (k, k + LP); iv is 1/D (last chunk, unscaled
    // residual) or -1/D (the scaled inner chunks' fused multiply-add).
    float2 za[LP], zb[LP], rr[LP], iv[LP], rs[LP];
    const int nxf = (gx + 1 < d.nx) + (gx > 0), nyf = (gy + 1 < d.ny) + (gy > 0);
#pragma unroll
    for (int k = 0; k < LP; ++k) {
      const int z0 = k, z1 = k + LP;
      if (!FIRST) {
        za[k] = make_float2(stage[z0 * SL + st], stage[z1 * SL + st]);
        zb[k] = make_float2(stage[(LMAX + z0) * SL + st], stage[(LMAX + z1) * SL + st]);
      }
      rr[k] = make_float2(stage[(2 * LMAX + z0) * SL + st], stage[(2 * LMAX + z1) * SL + st]);
      const float i0 = P.invd[nxf + 3 * nyf][z0], i1 = P.invd[nxf + 3 * nyf][z1];
      iv[k] = (SCALED && !LAST) ? make_float2(-i0, -i1) : make_float2(i0, i1);
      rs[k] = (SCALED && !LAST) ? make_float2(rr[k].x * i0, rr[k].y * i1) : rr[k];  // D^-1 r, fixed
      if (FIRST) {
        za[k] = SCALED ? make_float2(rr[k].x * i0 * P.z1s, rr[k].y * i1 * P.z1s)
                       : make_float2(rr[k].x * P.z1s, rr[k].y * P.z1s);
        zb[k] = make_float2(0.f, 0.f);
      }
    }
    __syncthreads();  // staging buffer consumed by every thread
    const int tn = t + gridDim.x;
    int txn = tx, tyn = ty;
    advance(txn, tyn);
    if (tid == 0 && tn < ntiles) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(txn, tyn);
    }
    // neighbour offsets inside a plane; a missing neighbour reads the cell itself
    const int oR = tid + ((gx + 1 < d.nx) ? 1 : 0), oL = tid - ((gx > 0) ? 1 : 0);
    const int oU = tid + ((gy + 1 < d.ny) ? TB_EX : 0), oD = tid - ((gy > 0) ? TB_EX : 0);
    const float2 m1 = make_float2(-1.f, -1.f);
    auto step = [&](const float2 (&C)[LP], float2 (&N)[LP], const int j) {
      float2* pl = reinterpret_cast<float2*>(plane) + (j & 1) * LP * PL;
#pragma unroll
      for (int k = 0; k < LP; ++k) pl[k * PL + tid] = C[k];
      __syncthreads();
      // rows outside the shrinking valid region skip the step as whole warps
      const bool upd = inside && ex > j && ex < TB_EX - 1 - j && ey > j && ey < EY - 1 - j;
      if (upd) {
#pragma unroll
        for (int k = 0; k < LP; ++k) {
          const float2 v = C[k];
          const float2* q = pl + k * PL;
          // per layer, in this order: d v, then the x pair, the y pair, the layer
          // above and the layer below (each lane rounds as the one-layer form would)
          float2 a = __fmul2_rn(P.d[k], v);
          a = __ffma2_rn(P.ngx[k], __fadd2_rn(q[oR], q[oL]), a);
          a = __ffma2_rn(P.ngy[k], __fadd2_rn(q[oU], q[oD]), a);
          if (k + 1 < LP) a = __ffma2_rn(P.ngzu[k], C[k + 1 < LP ? k + 1 : k], a);
          else a.x = fmaf(P.ngzu[k].x, C[0].y, a.x);  // layer LP - 1 below LP; the top layer has none
          if (k > 0) a = __ffma2_rn(P.ngzd[k], C[k > 0 ? k - 1 : k], a);
          else a.y = fmaf(P.ngzd[0].y, C[LP - 1].x, a.y);  // layer LP above LP - 1; layer 0 has none
          // the last chunk keeps r for z^T r and scales the residual instead
          const float2 res = !SCALED ? __ffma2_rn(a, m1, rr[k])
                                     : (LAST ? __fmul2_rn(__ffma2_rn(a, m1, rr[k]), iv[k])
                                             : __ffma2_rn(iv[k], a, rs[k]));
          N[k] = __ffma2_rn(P.c2[j], res, __ffma2_rn(P.c1[j], __ffma2_rn(N[k], m1, v), v));
        }
      }
    };
#pragma unroll
    for (int j = 0; j < STEPS; ++j) {
      if (j & 1) step(zb, za, j);
      else step(za, zb, j);
    }
    // the interior columns hold z_{m+STEPS} and z_{m+STEPS-1}
    const float2(&cur)[LP] = (STEPS & 1) ? zb : za;
    const float2(&prv)[LP] = (STEPS & 1) ? za : zb;
    const bool interior = inside && ex >= H && ex < H + TX && ey >= H && ey < H + TY;
    if (interior) {
      const long long base = (long long)gx + (long long)d.nx * gy;
#pragma unroll
      for (int z = 0; z < LMAX; ++z) {
        if (z < L) {
          const long long i = base + d.pxy * z;
          const int k = z < LP ? z : z - LP;
          const float c = z < LP ? cur[k].x : cur[k].y;
          out_cur[i] = c;
          if (out_prev) out_prev[i] = z < LP ? prv[k].x : prv[k].y;
          if (LAST) part[0] += (z < LP ? rr[k].x : rr[k].y) * c;
        }
      }
    }
    tx = txn;
    ty = tyn;
  }
  if (!LAST) return;
  double tot[1];
  if (!grid_reduce<float, 1>(part, partials, stride, counter, tot)) return;
  ctl->rz_next = tot[0];
  ctl_set_beta(ctl);
}

// ---------------------------------------------------------------------------
// Fused Chebyshev steps on grids with per-face conductances (a per-cell
// conductivity map): the same tile walk, staging pipeline and bounded waits as
// k_cheb_tb, with the face arrays staged beside the vectors.
//
// A tile is 32 x TBF_EY columns (768 threads, so a thread may hold 85 registers).
// Six boxes are staged per tile: z_m, z_{m-1}, r, gx, gy, gz.  Each thread keeps
// its column's own faces (+x, +y, +z per layer) and the face to the row below
// (-y) in registers; the face to the west (-x) is the west lane's +x face, taken by
// a warp shuffle.  The diagonal is summed once per tile in the one-step kernels'
// order (s, +x, -x, +y, -y, +z, -z) and inverted in FP32.  With the Jacobi
// scaling, D^-1 A v = v - D^-1 (sum_f g_f v_f) over the six neighbours f, so a
// step is
//   z_{m+1} = z_m + c1 (z_m - z_{m-1}) + c2 (D^-1 (r + sum_f g_f z_f) - z_m)
// (six products, no diagonal register).  Faces outside the grid are stored as 0;
// a missing neighbour is read as the cell itself and multiplied by that 0.
#define TBF_EY 24

template <int LMAX>
struct __align__(8) TBFParams {
  float2 c1[TB_H], c2[TB_H];  // Chebyshev step coefficients of this chunk, (c, c)
  float s[LMAX];             // per-layer diagonal term: h dx dy (top) + c dx dy dz / dt
  float z1s;                 // first chunk: z_1 = z1s D^-1 r
  int expire_test;           // test hook of the bounded wait (as in k_cheb_tb)
};

template <int LMAX>
constexpr size_t tbf_smem_bytes() {
  return ((size_t)6 * LMAX * TBF_EY * TB_BW + (size_t)2 * LMAX * TBF_EY * TB_EX) * sizeof(float) + 16 + 128;
}

template <int LMAX, int STEPS, bool LAST, bool FIRST>
__global__ void __launch_bounds__(TB_EX * TBF_EY, 1)
    k_cheb_tbf(Dims d, int ntx, int ntiles, int has_prev, Ctl* ctl, const __grid_constant__ CUtensorMap m_cur,
               const __grid_constant__ CUtensorMap m_prev, const __grid_constant__ CUtensorMap m_r,
               const __grid_constant__ CUtensorMap m_gx, const __grid_constant__ CUtensorMap m_gy,
               const __grid_constant__ CUtensorMap m_gz, const float* __restrict__ invd, float* __restrict__ out_cur,
               float* __restrict__ out_prev, const __grid_constant__ TBFParams<LMAX> P, double* partials, int stride,
               unsigned* counter) {
  if (ld_int(&ctl->done)) return;
  constexpr int EY = TBF_EY;
  constexpr int H = STEPS;
  constexpr int TX = TB_EX - 2 * H, TY = EY - 2 * H;  // interior of a tile
  static_assert(LMAX % 2 == 0, "layers are processed in pairs");
  constexpr int LP = LMAX / 2;
  constexpr int PL = EY * TB_EX;                        // floats per layer plane (float2 per pair plane)
  constexpr int SL = EY * TB_BW;                        // floats per staged layer
  extern __shared__ __align__(128) float tb_dyn[];
  float* tb_sm = tb_dyn + (((128u - (tb_smem(tb_dyn) & 127u)) & 127u) >> 2);  // 128-byte aligned
  float* stage = tb_sm;                  // [6][LMAX][EY][TB_BW]: z_m, z_{m-1}, r, gx, gy, gz
  float* plane = tb_sm + 6 * LMAX * SL;  // [2][LMAX][EY][TB_EX]
  unsigned long long* bar = (unsigned long long*)(plane + 2 * LMAX * PL);
  const int L = d.L;
  const int ex = threadIdx.x, ey = threadIdx.y;
  const int tid = ex + TB_EX * ey;
  const unsigned box_bytes = (unsigned)(L * SL * sizeof(float));
  const unsigned nbox = 4u + (FIRST ? 0u : (has_prev ? 2u : 1u));
  const unsigned tx_bytes = box_bytes * nbox;

  // staged layers the tensor copies never write (L..LMAX-1, and z_{m-1} when there
  // is none) are zeroed once
  for (int b = 0; b < 6; ++b) {
    const int z0 = (b == 1 && !has_prev) ? 0 : L;
    for (int i = tid; i < (LMAX - z0) * SL; i += TB_EX * EY) stage[(b * LMAX + z0) * SL + i] = 0.f;
  }
  if (tid == 0) {
    tb_mbar_init(bar, 1);
    tb_mbar_init(bar + 1, 1);  // test hook only: no thread ever arrives on it
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int tx, int ty) {
    const int xa = (tx * TX - H) & ~3, y0 = ty * TY - H;
    tb_mbar_expect(bar, tx_bytes);
    if (!FIRST) tb_tma_3d(stage, &m_cur, xa, y0, 0, bar);
    if (has_prev && !FIRST) tb_tma_3d(stage + LMAX * SL, &m_prev, xa, y0, 0, bar);
    tb_tma_3d(stage + 2 * LMAX * SL, &m_r, xa, y0, 0, bar);
    tb_tma_3d(stage + 3 * LMAX * SL, &m_gx, xa, y0, 0, bar);
    tb_tma_3d(stage + 4 * LMAX * SL, &m_gy, xa, y0, 0, bar);
    tb_tma_3d(stage + 5 * LMAX * SL, &m_gz, xa, y0, 0, bar);
  };
  const int dtx = (int)gridDim.x % ntx, dty = (int)gridDim.x / ntx;
  auto advance = [&](int& tx, int& ty) {
    tx += dtx;
    ty += dty;
    if (tx >= ntx) {
      tx -= ntx;
      ++ty;
    }
  };
  int tx = (int)blockIdx.x % ntx, ty = (int)blockIdx.x / ntx;
  if (tid == 0 && (int)blockIdx.x < ntiles) issue(tx, ty);

  float part[1] = {0.f};
  unsigned parity = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    bool ok = !(P.expire_test && t == (int)blockIdx.x) || tb_mbar_wait(bar + 1, 0u, TB_TEST_WAIT_NS);
    if (ok) ok = tb_mbar_wait(bar, parity);
    if (__syncthreads_or(!ok)) {
      // expiry: as in k_cheb_tb, record the error, end the loops and wait (bounded)
      // for this tile's copies before the CTA leaves
      if (tid == 0) {
        tb_mbar_wait(bar, parity);
        atomicCAS(&ctl->status, 0, 3);
        ctl->outer_done = 1;
        __threadfence();
        atomicExch(&ctl->done, 1);
      }
      break;
    }
    parity ^= 1u;
    const int x0 = tx * TX - H;
    const int gxi = x0 + ex;
    const int gyi = ty * TY - H + ey;
    const int st = ey * TB_BW + ex + (x0 - (x0 & ~3));  // this column in a staged layer
    const bool inside = gxi >= 0 && gxi < d.nx && gyi >= 0 && gyi < d.ny;
    // layer pairs (k, k + LP) as in k_cheb_tb: PR(a, z) is layer z of pair array a
    float2 za[LP], zb[LP], rr[LP], inv[LP], fx[LP], fy[LP], fyd[LP], fz[LP];
#define PR(a, z) ((z) < LP ? (a)[(z) < LP ? (z) : 0].x : (a)[(z) >= LP ? (z) - LP : 0].y)
#pragma unroll
    for (int z = 0; z < LMAX; ++z) {
      if (!FIRST) {
        PR(za, z) = stage[z * SL + st];
        PR(zb, z) = stage[(LMAX + z) * SL + st];
      }
      PR(rr, z) = stage[(2 * LMAX + z) * SL + st];
      PR(fx, z) = stage[(3 * LMAX + z) * SL + st];
      PR(fy, z) = stage[(4 * LMAX + z) * SL + st];
      PR(fyd, z) = ey > 0 ? stage[(4 * LMAX + z) * SL + st - TB_BW] : 0.f;
      PR(fz, z) = stage[(5 * LMAX + z) * SL + st];
    }
    // The diagonal in the one-step kernels' order: s, +x, -x, +y, -y, +z, -z.  A first
    // chunk forms z_1 = z1s D^-1 r on every column of the grown tile (step 0 reads the
    // outer ring too); the west ring (lane 0) and the south ring (row 0) lack the
    // staged -x / -y face, so they take 1/A_ii from the per-cell array.
    const bool ring = FIRST && (ex == 0 || ey == 0) && inside;
    const long long cbase = (long long)gxi + (long long)d.nx * gyi;
#pragma unroll
    for (int z = 0; z < LMAX; ++z) {
      const float fxz = PR(fx, z);
      const float fxw = __shfl_up_sync(0xffffffffu, fxz, 1);
      float dg = P.s[z];
      dg += fxz;
      dg += ex > 0 ? fxw : 0.f;
      dg += PR(fy, z);
      dg += PR(fyd, z);
      dg += PR(fz, z);
      dg += z > 0 ? PR(fz, z > 0 ? z - 1 : 0) : 0.f;
      float iv = 1.0f / dg;
      if (ring && z < L) iv = __ldg(invd + cbase + d.pxy * z);
      PR(inv, z) = (z < L && inside) ? iv : 0.f;  // columns outside the grid stay 0
      if (FIRST) {
        PR(za, z) = PR(rr, z) * PR(inv, z) * P.z1s;
        PR(zb, z) = 0.f;
      }
    }
#undef PR
    __syncthreads();  // staging buffer consumed by every thread
    const int tn = t + gridDim.x;
    int txn = tx, tyn = ty;
    advance(txn, tyn);
    if (tid == 0 && tn < ntiles) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(txn, tyn);
    }
    const int oR = tid + ((gxi + 1 < d.nx) ? 1 : 0), oL = tid - ((gxi > 0) ? 1 : 0);
    const int oU = tid + ((gyi + 1 < d.ny) ? TB_EX : 0), oD = tid - ((gyi > 0) ? TB_EX : 0);
    const float2 m1 = make_float2(-1.f, -1.f);
    auto step = [&](const float2 (&C)[LP], float2 (&N)[LP], const int j) {
      float2* pl = reinterpret_cast<float2*>(plane) + (j & 1) * LP * PL;
#pragma unroll
      for (int k = 0; k < LP; ++k) pl[k * PL + tid] = C[k];
      __syncthreads();
      const bool upd = inside && ex > j && ex < TB_EX - 1 - j && ey > j && ey < EY - 1 - j;
#pragma unroll
      for (int k = 0; k < LP; ++k) {
        // the west lane's +x faces (every lane: outside the branch)
        const float2 fxw = make_float2(__shfl_up_sync(0xffffffffu, fx[k].x, 1), __shfl_up_sync(0xffffffffu, fx[k].y, 1));
        if (upd) {
          const float2 v = C[k];
          const float2* q = pl + k * PL;
          // per layer: +x, -x, +y, -y, the layer above, the layer below
          float2 a = __fmul2_rn(fx[k], q[oR]);
          a = __ffma2_rn(fxw, q[oL], a);
          a = __ffma2_rn(fy[k], q[oU], a);
          a = __ffma2_rn(fyd[k], q[oD], a);
          if (k + 1 < LP) a = __ffma2_rn(fz[k], C[k + 1 < LP ? k + 1 : k], a);
          else a.x = fmaf(fz[k].x, C[0].y, a.x);  // layer LP - 1 below LP; the top layer has none
          if (k > 0) a = __ffma2_rn(fz[k > 0 ? k - 1 : k], C[k > 0 ? k - 1 : k], a);
          else a.y = fmaf(fz[LP - 1].x, C[LP - 1].x, a.y);  // layer LP above LP - 1; layer 0 has none
          const float2 res = __ffma2_rn(inv[k], __fadd2_rn(rr[k], a), __fmul2_rn(v, m1));  // D^-1 (r - A v)
          N[k] = __ffma2_rn(P.c2[j], res, __ffma2_rn(P.c1[j], __ffma2_rn(N[k], m1, v), v));
        }
      }
    };
#pragma unroll
    for (int j = 0; j < STEPS; ++j) {
      if (j & 1) step(zb, za, j);
      else step(za, zb, j);
    }
    const float2(&cur)[LP] = (STEPS & 1) ? zb : za;
    const float2(&prv)[LP] = (STEPS & 1) ? za : zb;
    const bool interior = inside && ex >= H && ex < H + TX && ey >= H && ey < H + TY;
    if (interior) {
      const long long base = (long long)gxi + (long long)d.nx * gyi;
#pragma unroll
      for (int z = 0; z < LMAX; ++z) {
        if (z < L) {
          const long long i = base + d.pxy * z;
          const int k = z < LP ? z : z - LP;
          const float c = z < LP ? cur[k].x : cur[k].y;
          out_cur[i] = c;
          if (out_prev) out_prev[i] = z < LP ? prv[k].x : prv[k].y;
          if (LAST) part[0] += (z < LP ? rr[k].x : rr[k].y) * c;
        }
      }
    }
    tx = txn;
    ty = tyn;
  }
  if (!LAST) return;
  double tot[1];
  if (!grid_reduce<float, 1>(part, partials, stride, counter, tot)) return;
  ctl->rz_next = tot[0];
  ctl_set_beta(ctl);
}
