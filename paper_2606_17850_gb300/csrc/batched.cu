// Batched steady solves of independent stacks in one persistent launch.
//
// Every instance is cut into tiles of 128 x 8 columns (all layers): the thread
// block of the vectorised z-walk kernels, 32 x 8 threads with 4 cells each.  All
// instances' tiles form one work list.  One cooperative kernel runs FP64 iterative
// refinement around FP32 PCG (Algorithm 1; Jacobi or Chebyshev preconditioner) for
// every instance: each phase (residual, search direction + stencil, update,
// Chebyshev step, ...) walks the tiles of the still-active instances, a grid-wide
// barrier separates phases, and one block per instance finishes that instance's
// reductions and takes its loop decisions with the same functions the single-grid
// kernels use.  An instance that has converged drops out of every later phase (its
// tiles are skipped); the loops end when no instance is active.
//
// Per tile, the block copies the instance descriptor and the loop scalars it needs
// into shared memory once (one L2 round trip), then the stencil phases run the
// z-walk engine of the single-grid kernels (per-layer coefficient table on grids
// with one conductivity per layer, per-face arrays otherwise).
//
// Vectors written during the kernel are read with ordinary (coherent) loads: the
// grid-wide barrier makes every write before it visible to every thread after it.
// Only immutable data (face conductances, tables, coefficients) uses the
// non-coherent read-only path (__ldg); control fields are read through L2 (__ldcg).
#include <cooperative_groups.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "internal.h"
#include "kernels_v4.cuh"
#include "mg_device.cuh"

namespace cg = cooperative_groups;

struct BInst {
  Dims d;
  int tile0, ntiles, tbx, uni;
  int rows;  // 8-row blocks per tile   } the tile shape the autotuner chose
  int zl;    // layers per tile           } for this instance's size class
  int tby;   // tiles along y
  Faces32 f32;
  Faces64 f64;
  const LayerTab* tab;
  const float* invd;
  const void* P;
  const double* T_in;  // initial guess (deg C) or NULL
  double* T_out;       // result (deg C)
  double t_amb;
  double* theta;
  float *r, *dv, *p[2], *mu, *zc[3];
  const float* c1;  // Chebyshev coefficients [k] (device)
  const float* c2;
  float inv_theta;
  Ctl* ctl;
};
static_assert(sizeof(BInst) % 4 == 0, "descriptor copied as 32-bit words");

struct BArgs {
  const BInst* inst;
  const int* tile_inst;
  int ninst, ntiles;
  double* partials;  // [2][ntiles]
  int pc, k, scaled;
  int max_sweeps;    // safety cap on inner sweeps of the whole batch
  // multigrid preconditioner (pc == TH_PC_MG): every instance's hierarchy, and for
  // each level index k the work list of 32 x 8-column tiles of the instances that
  // smooth on level k (entries [mgt_off[k], mgt_off[k+1]) of mgt: instance, tile).
  // The offsets live in device memory: an array member of this by-value argument
  // made ptxas keep the whole argument block on the stack (spill loads 292 -> 540
  // bytes in every instantiation, 0.93 -> 1.13 s for the 64-stack Chebyshev batch).
  const MGBDesc* mg;
  const int2* mgt;
  const int* mgt_off;  // [MG_BMAXL + 1]
  int mg_maxnl;
  const int2* mg_l0;  // per instance: first entry and count of its level-0 tiles
  double* mg_part;    // r^T z partial per level-0 tile
};

// loop scalars of one instance, read once per tile
struct BCtl {
  int act, first;
  float alpha, beta, rscale;
  double rnorm;
};

// Instance predicates (control fields change only in finish steps, between barriers).
enum { ACT_ALL = 0, ACT_OUTER = 1, ACT_INNER = 2 };
__device__ __forceinline__ bool active(const Ctl* c, int what) {
  if (what == ACT_ALL) return true;
  if (what == ACT_OUTER) return __ldcg(&c->outer_done) == 0;
  return __ldcg(&c->outer_done) == 0 && __ldcg(&c->done) == 0;
}

// Any instance active (every block computes the same answer after a barrier).
__device__ bool any_active(const BArgs& A, int what) {
  __shared__ int flag;
  if (thread_linear_id() == 0) {
    int f = 0;
    for (int j = 0; j < A.ninst && !f; ++j) f = active(A.inst[j].ctl, what);
    flag = f;
  }
  __syncthreads();
  const bool r = flag != 0;
  __syncthreads();
  return r;
}

// row block rb (0 <= rb < I.rows) of tile t: 128 x 8 columns, layers [zs, ze)
__device__ __forceinline__ Walk4 tile_walk(const BInst& I, int t, int rb) {
  const int loc = t - I.tile0;
  const int bx = loc % I.tbx, by = (loc / I.tbx) % I.tby, bz = loc / (I.tbx * I.tby);
  Walk4 w;
  w.x0 = 4 * (bx * TH_BX + threadIdx.x);
  w.y = (by * I.rows + rb) * TH_BY4 + threadIdx.y;
  w.zs = bz * I.zl;
  w.ze = min(w.zs + I.zl, I.d.L);
  w.valid = (w.x0 < I.d.nx) && (w.y < I.d.ny);
  w.b0 = (long long)w.x0 + (long long)I.d.nx * w.y;
  return w;
}

// One phase over the active instances' tiles: body(I, C, w, v) with the tile's
// instance I and loop scalars C in shared memory fills NQ per-thread partial sums,
// reduced per tile into partials[q][t].  The loop scalars change only in finish
// steps (between grid barriers), so within a phase the descriptor and scalars of an
// instance are copied once and kept while the block's next tiles belong to the same
// instance.
template <int NQ, class F>
__device__ void phase(const BArgs& A, int what, F body) {
  __shared__ BInst si;
  __shared__ BCtl sc;
  __shared__ double sm[2][32];
  const int tid = thread_linear_id(), nw = (block_threads() + 31) >> 5;
  int cur = -1;
  for (int t = blockIdx.x; t < A.ntiles; t += gridDim.x) {
    const int ii = __ldg(A.tile_inst + t);
    if (ii != cur) {
      __syncthreads();  // the previous instance's descriptor and scalars are no longer read
      const int* src = reinterpret_cast<const int*>(A.inst + ii);
      int* dst = reinterpret_cast<int*>(&si);
      for (int q = tid; q < (int)(sizeof(BInst) / 4); q += block_threads()) dst[q] = __ldg(src + q);
      if (tid == 0) {
        const Ctl* c = A.inst[ii].ctl;
        sc.act = active(c, what);
        sc.first = __ldcg(&c->first);
        sc.alpha = __ldcg(&c->alpha_f);
        sc.beta = __ldcg(&c->beta_f);
        sc.rscale = __ldcg(&c->rscale_f);
        sc.rnorm = __ldcg(&c->rnorm);
      }
      __syncthreads();
      cur = ii;
    }
    if (sc.act) {
      float v[NQ > 0 ? NQ : 1] = {};
      for (int rb = 0; rb < si.rows; ++rb) {
        const Walk4 w = tile_walk(si, t, rb);
        if (w.valid) body(si, sc, w, v);
      }
      if (NQ > 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const float s = warp_sum(v[q]);
          if ((tid & 31) == 0) sm[q][tid >> 5] = (double)s;
        }
        __syncthreads();
        if (tid == 0) {
#pragma unroll
          for (int q = 0; q < NQ; ++q) {
            double s = 0.0;
            for (int w2 = 0; w2 < nw; ++w2) s += sm[q][w2];
            A.partials[(size_t)q * A.ntiles + t] = s;
          }
        }
        __syncthreads();  // sm is rewritten by the next tile's reduction
      }
    }
  }
  __syncthreads();  // the next phase's blocks may reuse this block's shared memory
}

// One block per active instance sums its tiles' partials (fixed order) and runs fin.
template <int NQ, class F>
__device__ void finish(const BArgs& A, int what, F fin) {
  __shared__ double sm[2][32];
  const int tid = thread_linear_id(), nw = (block_threads() + 31) >> 5;
  for (int j = blockIdx.x; j < A.ninst; j += gridDim.x) {
    const BInst& I = A.inst[j];
    if (!active(I.ctl, what)) continue;
    double s[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      s[q] = 0.0;
      for (int t = I.tile0 + tid; t < I.tile0 + I.ntiles; t += block_threads())
        s[q] += __ldcg(A.partials + (size_t)q * A.ntiles + t);
      s[q] = warp_sum(s[q]);
      if ((tid & 31) == 0) sm[q][tid >> 5] = s[q];
    }
    __syncthreads();
    if (tid == 0) {
      double tot[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        tot[q] = 0.0;
        for (int w = 0; w < nw; ++w) tot[q] += sm[q][w];
      }
      fin(I.ctl, tot);
    }
    __syncthreads();
  }
}

// the layers of a tile column segment: f(i) for i = index of its first cell in each layer
template <class F>
__device__ __forceinline__ void for_layers(const BInst& I, const Walk4& w, F f) {
  for (int z = w.zs; z < w.ze; ++z) f(w.b0 + (long long)z * I.d.pxy, z);
}

// FP64 refinement residual r = P - A theta of 4 cells per layer, and ||r||^2, ||P||^2
template <typename TP>
__device__ void body_residual(const BInst& I, const Walk4& w, float (&v)[2]) {
  for_layers(I, w, [&](long long i0, int z) {
    const double s = __ldg(&I.tab->s64[z]);
    float o[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      Cell c;
      c.x = w.x0 + k;
      c.y = w.y;
      c.z = z;
      c.i = i0 + k;
      c.valid = true;
      double dg;
      const double ti = I.theta[c.i];
      const double a = stencil_row<double>(I.f64.gx, I.f64.gy, I.f64.gz, I.d, c, s, ti,
                                           [&](long long j) { return I.theta[j]; }, dg);
      const double b = (double)((const TP*)I.P)[c.i];
      const float rf = (float)(b - a), bf = (float)b;
      o[k] = rf;
      v[0] += rf * rf;
      v[1] += bf * bf;
    }
    st4(I.r + i0, make_float4(o[0], o[1], o[2], o[3]));
  });
}

// z for the Jacobi / first Chebyshev iterate / none, 4 cells
__device__ __forceinline__ float4 z_of4(const BArgs& A, const BInst& I, long long i, const float4& r) {
  if (A.pc == TH_PC_NONE) return r;
  float4 z = r;
  if (A.pc == TH_PC_JACOBI || A.scaled) {
    const float4 iv = __ldg(reinterpret_cast<const float4*>(I.invd + i));
    z = make_float4(r.x * iv.x, r.y * iv.y, r.z * iv.z, r.w * iv.w);
  }
  if (A.pc == TH_PC_CHEB) z = make_float4(z.x * I.inv_theta, z.y * I.inv_theta, z.z * I.inv_theta, z.w * I.inv_theta);
  return z;
}

__device__ __forceinline__ float dot4(const float4& a, const float4& b) {
  return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}

// stencil walk over a tile with the instance's coefficient source
template <typename F4, typename F1, typename E>
__device__ __forceinline__ void walk(const BInst& I, const Walk4& w, F4 V4, F1 V1, E epi) {
  if (I.uni)
    zwalk4<float, true>(I.d, w, I.f32.gx, I.f32.gy, I.f32.gz, I.tab, V4, V1, epi);
  else
    zwalk4<float, false>(I.d, w, I.f32.gx, I.f32.gy, I.f32.gz, I.tab, V4, V1, epi);
}

__device__ void cheb_tail(const BArgs& A, cg::grid_group& grid) {
  for (int m = 1; m < A.k; ++m) {
    const bool last = (m == A.k - 1);
    phase<1>(A, ACT_INNER, [&](const BInst& I, const BCtl&, const Walk4& w, float (&v)[1]) {
      const float* zprev = (m >= 2) ? I.zc[(m - 2) % 3] : nullptr;
      const float* zcur = I.zc[(m - 1) % 3];
      float* znext = I.zc[m % 3];
      const float c1 = __ldg(I.c1 + m), c2 = __ldg(I.c2 + m);
      walk(I, w, [&](long long i) { return ld4(zcur + i); }, [&](long long j) { return zcur[j]; },
           [&](long long i, int, const float4& zv, const float (&acc)[4], const float (&dg)[4]) {
             const float4 rv = ld4(I.r + i);
             const float4 zp = zprev ? ld4(zprev + i) : z4();
             float o[4];
#pragma unroll
             for (int k = 0; k < 4; ++k) {
               const float zk = cmp(zv, k);
               float res = cmp(rv, k) - acc[k];
               if (A.scaled) res = res / dg[k];
               o[k] = zk + c1 * (zk - cmp(zp, k)) + c2 * res;
               if (last) v[0] += cmp(rv, k) * o[k];
             }
             st4(znext + i, make_float4(o[0], o[1], o[2], o[3]));
           });
    });
    grid.sync();
    if (last) {
      finish<1>(A, ACT_INNER, [&](Ctl* ctl, const double (&t)[1]) {
        ctl->rz_next = t[0];
        ctl_set_beta(ctl);
      });
      grid.sync();
    }
  }
}

// ---------------------------------------------------------------- multigrid phases

// placeholder table for the per-cell variant of the level routines (levels without a
// layer-uniform table read their per-cell arrays; the table argument is unused there)
static __constant__ MGUni<8> c_mg_none;

// One phase over the level-k tile list: body(instance, tile within its level, entry)
// for the tiles of instances whose inner solve is active (checked once per instance
// run, the flag cannot change within a phase).
template <class F>
__device__ void mg_phase(const BArgs& A, int k, F body) {
  __shared__ int s_act;
  const int tid = thread_linear_id();
  int cur = -1;
  bool act = false;
  const int t0 = __ldg(A.mgt_off + k), t1 = __ldg(A.mgt_off + k + 1);
  for (int t = t0 + (int)blockIdx.x; t < t1; t += gridDim.x) {
    const int2 e = __ldg(A.mgt + t);
    if (e.x != cur) {
      __syncthreads();
      if (tid == 0) s_act = active(A.inst[e.x].ctl, ACT_INNER);
      __syncthreads();
      act = s_act != 0;
      cur = e.x;
    }
    if (act) body(e.x, e.y, t);
  }
  __syncthreads();
}

__device__ __forceinline__ MGDev mg_dev(const MGBDesc& D, int k, int L) {
  const MGBLevel& l = D.lv[k];
  return MGDev{l.nx, l.ny, L, l.gx, l.gy, l.gz, l.s, l.m, l.w};
}

// z = M^-1 r for every active instance: one V-cycle (as mg_vcycle of the single-grid
// path), instances of different depths in the same phases; the last post-smoothing
// also reduces r^T z.  Inlined (the multigrid instantiation spills about 1.1 KB a
// thread, yet measured faster than the cycle as an out-of-line call, 314 vs 330 ms
// for the 64 stacks, or at two blocks per SM without the register cap, 414 ms).
__device__ void mg_vcycle_batched(const BArgs& A, cg::grid_group& grid) {
  __shared__ float rowsum[8][32];
  __shared__ double red[32];
  const int tid = thread_linear_id();
  for (int k = 0; k + 1 < A.mg_maxnl; ++k) {  // down: pre-smooth from zero, restrict
    mg_phase(A, k, [&](int ii, int tile, int) {
      const MGBDesc& D = A.mg[ii];
      const BInst& I = A.inst[ii];
      const MGBLevel& l = D.lv[k];
      const int tbx = (l.nx + 31) / 32;
      const int x = (tile % tbx) * 32 + threadIdx.x, y = (tile / tbx) * 8 + threadIdx.y;
      const float* b = (k == 0) ? I.r : l.b;
      float* xo = (k == 0) ? l.xt : l.x;
      if (x < l.nx && y < l.ny) {
        if (l.uni)
          mg_smooth_column<8, true>(mg_dev(D, k, I.d.L), l.t, x, y, b, nullptr, nullptr, 1, 1, xo, kMGOmega, false);
        else
          mg_smooth_column<8, false>(mg_dev(D, k, I.d.L), c_mg_none, x, y, b, nullptr, nullptr, 1, 1, xo, kMGOmega,
                                     false);
      }
    });
    grid.sync();
    mg_phase(A, k, [&](int ii, int tile, int) {
      const MGBDesc& D = A.mg[ii];
      const BInst& I = A.inst[ii];
      const MGBLevel& l = D.lv[k];
      const MGBLevel& c = D.lv[k + 1];
      const int tbx = (l.nx + 31) / 32;
      if (l.uni)
        mg_restrict_tile<8, true>(mg_dev(D, k, I.d.L), l.t, tile % tbx, tile / tbx, (k == 0) ? I.r : l.b,
                                  (k == 0) ? l.xt : l.x, c.nx, c.ny, c.b, rowsum);
      else
        mg_restrict_tile<8, false>(mg_dev(D, k, I.d.L), c_mg_none, tile % tbx, tile / tbx, (k == 0) ? I.r : l.b,
                                   (k == 0) ? l.xt : l.x, c.nx, c.ny, c.b, rowsum);
    });
    grid.sync();
  }
  // coarsest level of every active instance: the dense solve, one block at a time
  {
    int cur = -1;
    for (int j = blockIdx.x; j < A.ninst; j += gridDim.x) {
      if (!active(A.inst[j].ctl, ACT_INNER)) continue;
      const MGBDesc& D = A.mg[j];
      const MGBLevel& c = D.lv[D.nl - 1];
      mg_coarsest_rows(D.nc, D.cinv, c.b, c.x, tid >> 5, block_threads() >> 5);
      cur = j;
    }
    (void)cur;
  }
  grid.sync();
  for (int k = A.mg_maxnl - 2; k >= 0; --k) {  // up: prolongated correction + post-smooth
    mg_phase(A, k, [&](int ii, int tile, int t) {
      const MGBDesc& D = A.mg[ii];
      const BInst& I = A.inst[ii];
      const MGBLevel& l = D.lv[k];
      const MGBLevel& c = D.lv[k + 1];
      const int tbx = (l.nx + 31) / 32;
      const int x = (tile % tbx) * 32 + threadIdx.x, y = (tile / tbx) * 8 + threadIdx.y;
      const float* b = (k == 0) ? I.r : l.b;
      const float* xin = (k == 0) ? l.xt : l.x;
      const float* xc = (k + 1 == D.nl - 1) ? c.x : c.xt;
      float* out = (k == 0) ? I.zc[0] : l.xt;
      float rz = 0.f;
      if (x < l.nx && y < l.ny) {
        if (l.uni)
          rz = mg_smooth_column<8, true>(mg_dev(D, k, I.d.L), l.t, x, y, b, xin, xc, c.nx, c.ny, out, kMGOmega,
                                         k == 0);
        else
          rz = mg_smooth_column<8, false>(mg_dev(D, k, I.d.L), c_mg_none, x, y, b, xin, xc, c.nx, c.ny, out,
                                          kMGOmega, k == 0);
      }
      if (k == 0) {  // r^T z of the tile
        const float ws = warp_sum(rz);
        if ((tid & 31) == 0) red[tid >> 5] = (double)ws;
        __syncthreads();
        if (tid == 0) {
          double sum = 0.0;
          for (int w = 0; w < (block_threads() >> 5); ++w) sum += red[w];
          A.mg_part[t - __ldg(A.mgt_off)] = sum;
        }
        __syncthreads();
      }
    });
    grid.sync();
  }
  // r^T z per instance (fixed order), then beta
  for (int j = blockIdx.x; j < A.ninst; j += gridDim.x) {
    const Ctl* c0 = A.inst[j].ctl;
    if (!active(c0, ACT_INNER)) continue;
    const int2 rg = __ldg(A.mg_l0 + j);
    double sum = 0.0;
    for (int q = rg.x + tid; q < rg.x + rg.y; q += block_threads()) sum += __ldcg(A.mg_part + q);
    sum = warp_sum(sum);
    if ((tid & 31) == 0) red[tid >> 5] = sum;
    __syncthreads();
    if (tid == 0) {
      double tot = 0.0;
      for (int w = 0; w < (block_threads() >> 5); ++w) tot += red[w];
      Ctl* ctl = A.inst[j].ctl;
      ctl->rz_next = tot;
      ctl_set_beta(ctl);
    }
    __syncthreads();
  }
  grid.sync();
}

// Three co-resident blocks per SM (at most 80 registers a thread): the memory-bound
// phases need the occupancy more than the rarely run FP64 residual phase needs
// registers (measured: 0.92 s vs 1.12 s with two blocks per SM for the 64 stacks).
// MGP: the multigrid instantiation (its V-cycle phases are compiled only there, so
// the other preconditioners keep their register allocation)
template <typename TP, bool MGP>
__global__ void __launch_bounds__(TH_BX* TH_BY4, 3) k_batched(BArgs A) {
  cg::grid_group grid = cg::this_grid();
  const int rz_here = (A.pc == TH_PC_NONE || A.pc == TH_PC_JACOBI || (A.pc == TH_PC_CHEB && A.k == 1)) ? 1 : 0;
  auto zfinal = [&](const BInst& I) -> const float* {
    if (A.pc == TH_PC_NONE) return I.r;
    if (A.pc == TH_PC_CHEB) return I.zc[(A.k - 1) % 3];
    return I.zc[0];
  };
  // theta from the initial guess
  phase<0>(A, ACT_ALL, [&](const BInst& I, const BCtl&, const Walk4& w, float (&)[1]) {
    for_layers(I, w, [&](long long i0, int) {
#pragma unroll
      for (int k = 0; k < 4; ++k) I.theta[i0 + k] = I.T_in ? I.T_in[i0 + k] - I.t_amb : 0.0;
    });
  });
  grid.sync();
  phase<2>(A, ACT_OUTER, [&](const BInst& I, const BCtl&, const Walk4& w, float (&v)[2]) {
    body_residual<TP>(I, w, v);
  });
  grid.sync();
  finish<2>(A, ACT_OUTER, [&](Ctl* ctl, const double (&t)[2]) { fin_residual(ctl, t[0], t[1], 0, 0); });
  grid.sync();
  int sweeps = 0;
  while (any_active(A, ACT_OUTER)) {
    // start of an inner solve: r scaled to unit norm, d = 0, z_0 = M r
    phase<2>(A, ACT_OUTER, [&](const BInst& I, const BCtl& C, const Walk4& w, float (&v)[2]) {
      for_layers(I, w, [&](long long i, int) {
        float4 r = ld4(I.r + i);
        r = make_float4(r.x * C.rscale, r.y * C.rscale, r.z * C.rscale, r.w * C.rscale);
        st4(I.r + i, r);
        st4(I.dv + i, z4());
        v[0] += dot4(r, r);
        if (!MGP) {  // multigrid: z and r^T z come from the V-cycle
          const float4 z = z_of4(A, I, i, r);
          if (A.pc != TH_PC_NONE) st4(I.zc[0] + i, z);
          v[1] += dot4(r, z);
        }
      });
    });
    grid.sync();
    finish<2>(A, ACT_OUTER, [&](Ctl* ctl, const double (&t)[2]) { fin_update(ctl, t[0], t[1], true, rz_here); });
    grid.sync();
    if (A.pc == TH_PC_CHEB) cheb_tail(A, grid);
    if (MGP) mg_vcycle_batched(A, grid);
    int parity = 0;
    while (any_active(A, ACT_INNER) && sweeps < A.max_sweeps) {
      ++sweeps;
      // p_new = z + beta p_old, mu = A p_new, p^T mu
      phase<1>(A, ACT_INNER, [&](const BInst& I, const BCtl& C, const Walk4& w, float (&v)[1]) {
        const float* z = zfinal(I);
        const float* po = I.p[parity];
        float* pn = I.p[1 - parity];
        const int first = C.first;
        const float beta = first ? 0.f : C.beta;
        auto P4 = [&](long long i) -> float4 {
          const float4 a = ld4(z + i);
          if (first) return a;
          const float4 b = ld4(po + i);
          return make_float4(a.x + beta * b.x, a.y + beta * b.y, a.z + beta * b.z, a.w + beta * b.w);
        };
        auto P1 = [&](long long j) -> float { return first ? z[j] : z[j] + beta * po[j]; };
        walk(I, w, P4, P1, [&](long long i, int, const float4& pv, const float (&acc)[4], const float (&)[4]) {
          st4(pn + i, pv);
          st4(I.mu + i, make_float4(acc[0], acc[1], acc[2], acc[3]));
#pragma unroll
          for (int k = 0; k < 4; ++k) v[0] += cmp(pv, k) * acc[k];
        });
      });
      grid.sync();
      finish<1>(A, ACT_INNER, [&](Ctl* ctl, const double (&t)[1]) { fin_pap(ctl, t[0]); });
      grid.sync();
      // d += alpha p, r -= alpha mu, z = M r
      phase<2>(A, ACT_INNER, [&](const BInst& I, const BCtl& C, const Walk4& w, float (&v)[2]) {
        const float alpha = C.alpha;
        const float* pn = I.p[1 - parity];
        for_layers(I, w, [&](long long i, int) {
          const float4 d = ld4(I.dv + i), p = ld4(pn + i), m = ld4(I.mu + i);
          float4 r = ld4(I.r + i);
          st4(I.dv + i, make_float4(d.x + alpha * p.x, d.y + alpha * p.y, d.z + alpha * p.z, d.w + alpha * p.w));
          r = make_float4(r.x - alpha * m.x, r.y - alpha * m.y, r.z - alpha * m.z, r.w - alpha * m.w);
          st4(I.r + i, r);
          v[0] += dot4(r, r);
          if (!MGP) {
            const float4 z = z_of4(A, I, i, r);
            if (A.pc != TH_PC_NONE) st4(I.zc[0] + i, z);
            v[1] += dot4(r, z);
          }
        });
      });
      grid.sync();
      finish<2>(A, ACT_INNER, [&](Ctl* ctl, const double (&t)[2]) { fin_update(ctl, t[0], t[1], false, rz_here); });
      grid.sync();
      if (A.pc == TH_PC_CHEB) cheb_tail(A, grid);
      if (MGP) mg_vcycle_batched(A, grid);
      parity ^= 1;
    }
    // theta += ||r|| d, then the true FP64 residual decides the outer loop
    phase<0>(A, ACT_OUTER, [&](const BInst& I, const BCtl& C, const Walk4& w, float (&)[1]) {
      for_layers(I, w, [&](long long i0, int) {
        const float4 d = ld4(I.dv + i0);
#pragma unroll
        for (int k = 0; k < 4; ++k) I.theta[i0 + k] += C.rnorm * (double)cmp(d, k);
      });
    });
    grid.sync();
    phase<2>(A, ACT_OUTER, [&](const BInst& I, const BCtl&, const Walk4& w, float (&v)[2]) {
      body_residual<TP>(I, w, v);
    });
    grid.sync();
    finish<2>(A, ACT_OUTER, [&](Ctl* ctl, const double (&t)[2]) { fin_residual(ctl, t[0], t[1], 0, 1); });
    grid.sync();
    if (sweeps >= A.max_sweeps) break;
  }
  phase<0>(A, ACT_ALL, [&](const BInst& I, const BCtl&, const Walk4& w, float (&)[1]) {
    for_layers(I, w, [&](long long i0, int) {
#pragma unroll
      for (int k = 0; k < 4; ++k) I.T_out[i0 + k] = I.theta[i0 + k] + I.t_amb;
    });
  });
}

// ------------------------------------------------------------------ host

template <typename T>
struct DevArr {
  T* p = nullptr;
  ~DevArr() {
    if (p) cudaFree(p);
  }
  th_status alloc(size_t n) {
    if (cudaMalloc((void**)&p, sizeof(T) * (n ? n : 1)) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return th_fail(TH_ENOMEM, "batched workspace allocation failed");
    }
    return TH_OK;
  }
};

static th_status sequential(thermal_grid* const* grids, int n, const void* const* power, int power_dtype,
                            double* const* T, const thermal_solve_opts* opts, thermal_solve_stats* stats,
                            cudaStream_t s) {
  th_status first_bad = TH_OK;
  std::string first_msg;
  for (int i = 0; i < n; ++i) {
    thermal_solve_stats st;
    std::memset(&st, 0, sizeof(st));
    const void* maps[1] = {power[i]};
    th_status r = solver_drive(grids[i], KIND_STEADY, 0.0, maps, 1, power_dtype, 1, 1, T[i], opts, &st, s);
    st.status = r;
    if (stats) stats[i] = st;
    if (r != TH_OK && first_bad == TH_OK) {
      first_bad = r;
      first_msg = thermal_last_error();
    }
    if (r == TH_ECUDA) break;
  }
  if (first_bad != TH_OK) return th_fail(first_bad, "%s", first_msg.c_str());
  return TH_OK;
}

// Control block of one instance at the start of a batched solve.
static Ctl batch_ctl(const thermal_solve_opts* o, double tol, int max_outer, int max_inner) {
  Ctl c;
  std::memset(&c, 0, sizeof(c));
  c.tol_rel = tol;
  c.inner_tol = o->inner_tol;
  c.inner_rel = o->inner_tol;
  c.max_outer = max_outer;
  c.max_inner = max_inner;
  c.n_steps = 1;
  c.steps_per_map = 1;
  c.n_maps = 1;
  c.rel_res = 1.0;
  return c;
}

// One cooperative launch of the persistent kernel over the instances hi (tile lists
// built from each instance's row blocks per tile); *ms = its duration (CUDA events).
// mgd (multigrid preconditioner only): each instance's hierarchy, aligned with hi
static th_status launch_batch(std::vector<BInst>& hi, const std::vector<thermal_grid*>& gs, const Ctl* ctl0,
                              int power_dtype, const thermal_solve_opts* opts, int k, int max_sweeps,
                              cudaStream_t s, float* ms, const std::vector<MGBDesc>* mgd = nullptr) {
  const int n = (int)hi.size();
  std::vector<int> tile_inst;
  int ntiles = 0;
  for (int i = 0; i < n; ++i) {
    BInst& I = hi[i];
    I.tbx = (I.d.nx + 4 * TH_BX - 1) / (4 * TH_BX);
    I.tby = (I.d.ny + TH_BY4 * I.rows - 1) / (TH_BY4 * I.rows);
    I.tile0 = ntiles;
    I.ntiles = I.tbx * I.tby * ((I.d.L + I.zl - 1) / I.zl);
    ntiles += I.ntiles;
    for (int t = 0; t < I.ntiles; ++t) tile_inst.push_back(i);
    TH_CUDA(cudaMemcpyAsync(gs[i]->ctl, &ctl0[i], sizeof(Ctl), cudaMemcpyHostToDevice, s));
  }
  DevArr<BInst> dinst;
  DevArr<int> dtiles;
  DevArr<double> dpart;
  TH_TRY(dinst.alloc(n));
  TH_TRY(dtiles.alloc(ntiles));
  TH_TRY(dpart.alloc((size_t)2 * ntiles));
  TH_CUDA(cudaMemcpyAsync(dinst.p, hi.data(), sizeof(BInst) * n, cudaMemcpyHostToDevice, s));
  TH_CUDA(cudaMemcpyAsync(dtiles.p, tile_inst.data(), sizeof(int) * ntiles, cudaMemcpyHostToDevice, s));
  BArgs A;
  A.inst = dinst.p;
  A.tile_inst = dtiles.p;
  A.ninst = n;
  A.ntiles = ntiles;
  A.partials = dpart.p;
  A.pc = opts->precond;
  A.k = k;
  A.scaled = opts->cheb_scaled ? 1 : 0;
  A.max_sweeps = max_sweeps;
  // multigrid: per level index, the 32 x 8-column tiles of the instances that smooth
  // on that level (instance by instance, so each instance's level-0 tiles are one range)
  DevArr<MGBDesc> dmg;
  DevArr<int2> dmgt, dml0;
  DevArr<int> dmgo;
  DevArr<double> dmgp;
  A.mg = nullptr;
  A.mgt = nullptr;
  A.mgt_off = nullptr;
  A.mg_l0 = nullptr;
  A.mg_part = nullptr;
  A.mg_maxnl = 0;
  if (opts->precond == TH_PC_MG) {
    if (!mgd || (int)mgd->size() != n) return th_fail(TH_ESTATE, "batched multigrid without hierarchies");
    int maxnl = 0;
    for (const MGBDesc& D : *mgd) maxnl = std::max(maxnl, D.nl);
    std::vector<int2> lst;
    std::vector<int2> l0(n, make_int2(0, 0));
    std::vector<int> off(MG_BMAXL + 1, 0);
    for (int lvl = 0; lvl + 1 < maxnl; ++lvl) {
      off[lvl] = (int)lst.size();
      for (int i = 0; i < n; ++i) {
        const MGBDesc& D = (*mgd)[i];
        if (lvl > D.nl - 2) continue;
        const int nt = ((D.lv[lvl].nx + 31) / 32) * ((D.lv[lvl].ny + 7) / 8);
        if (lvl == 0) l0[i] = make_int2((int)lst.size(), nt);
        for (int t = 0; t < nt; ++t) lst.push_back(make_int2(i, t));
      }
    }
    for (int lvl = std::max(maxnl - 1, 0); lvl <= MG_BMAXL; ++lvl) off[lvl] = (int)lst.size();
    TH_TRY(dmg.alloc(n));
    TH_TRY(dmgt.alloc(lst.size()));
    TH_TRY(dmgo.alloc(off.size()));
    TH_TRY(dml0.alloc(n));
    TH_TRY(dmgp.alloc(std::max(1, off[1] - off[0])));
    TH_CUDA(cudaMemcpyAsync(dmg.p, mgd->data(), sizeof(MGBDesc) * n, cudaMemcpyHostToDevice, s));
    if (!lst.empty())
      TH_CUDA(cudaMemcpyAsync(dmgt.p, lst.data(), sizeof(int2) * lst.size(), cudaMemcpyHostToDevice, s));
    TH_CUDA(cudaMemcpyAsync(dml0.p, l0.data(), sizeof(int2) * n, cudaMemcpyHostToDevice, s));
    TH_CUDA(cudaMemcpyAsync(dmgo.p, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice, s));
    A.mg = dmg.p;
    A.mgt = dmgt.p;
    A.mgt_off = dmgo.p;
    A.mg_l0 = dml0.p;
    A.mg_part = dmgp.p;
    A.mg_maxnl = maxnl;
  }
  // co-resident grid: every block must be resident for the grid-wide barriers
  int dev = 0, sms = 0, per_sm = 0;
  TH_CUDA(cudaGetDevice(&dev));
  TH_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  void* fn = opts->precond == TH_PC_MG
                 ? (power_dtype == TH_F64 ? (void*)k_batched<double, true> : (void*)k_batched<float, true>)
                 : (power_dtype == TH_F64 ? (void*)k_batched<double, false> : (void*)k_batched<float, false>);
  TH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, TH_BX * TH_BY4, 0));
  if (per_sm < 1) return th_fail(TH_ECUDA, "batched kernel cannot be resident");
  const int nblocks = std::max(1, std::min(ntiles, sms * per_sm));
  void* args[] = {&A};
  cudaEvent_t e0, e1;
  TH_CUDA(cudaEventCreate(&e0));
  TH_CUDA(cudaEventCreate(&e1));
  struct EvGuard { cudaEvent_t a, b; ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); } } eg{e0, e1};
  TH_CUDA(cudaEventRecord(e0, s));
  TH_CUDA(cudaLaunchCooperativeKernel(fn, dim3(nblocks), dim3(TH_BX, TH_BY4), args, 0, s));
  TH_CUDA(cudaEventRecord(e1, s));
  TH_CUDA(cudaStreamSynchronize(s));
  TH_CUDA(cudaEventElapsedTime(ms, e0, e1));
  return TH_OK;
}

// Tile autotuner: the tile shape of each size class (nx, ny, layers, coefficient
// source) and preconditioner, chosen once per process by timing a fixed amount of work (one refinement
// step with three inner iterations, from theta = 0) on the batch's instances of the
// class, launched together as in the real solve, with each candidate: row blocks per tile (1 or 2 blocks of 128 x 8 columns) times
// layers per tile (all, half, a quarter).  More rows or layers per tile mean fewer
// tiles and fewer per-tile descriptor copies; fewer layers per thread mean more
// threads with loads in flight (the z-walk keeps the layer below and above in
// registers, so a layer chunk re-reads one plane at each end).
struct BClass {
  int nx, ny, L, uni, pc, k;  // the preconditioner's phases weigh differently
  bool operator<(const BClass& o) const {
    return std::tie(nx, ny, L, uni, pc, k) < std::tie(o.nx, o.ny, o.L, o.uni, o.pc, o.k);
  }
};
struct BShape { int rows, zc; };
static std::mutex g_rows_mu;
static std::map<BClass, BShape> g_rows;

static th_status tune_rows(std::vector<BInst>& hi, const std::vector<thermal_grid*>& gs, int power_dtype,
                           const thermal_solve_opts* opts, int k, cudaStream_t s,
                           const std::vector<MGBDesc>* mgd) {
  // instances of each size class in this batch
  std::map<BClass, std::vector<size_t>> classes;
  for (size_t i = 0; i < hi.size(); ++i)
    classes[BClass{hi[i].d.nx, hi[i].d.ny, hi[i].d.L, hi[i].uni, opts->precond, k}].push_back(i);
  for (auto& kv : classes) {
    const BClass& key = kv.first;
    const std::vector<size_t>& members = kv.second;
    BShape chosen{1, key.L};
    bool cached = false;
    {
      std::lock_guard<std::mutex> lk(g_rows_mu);
      auto it = g_rows.find(key);
      if (it != g_rows.end()) {
        chosen = it->second;
        cached = true;
      }
    }
    if (!cached) {
      const int L = key.L;
      std::vector<BShape> cand;
      for (int r : {1, 2})
        for (int zl : {L, (L + 1) / 2, (L + 3) / 4}) {
          if (r > 1 && (key.ny + TH_BY4 - 1) / TH_BY4 < r) continue;  // taller than the grid
          bool dup = false;
          for (const BShape& c : cand) dup = dup || (c.rows == r && c.zc == zl);
          if (!dup) cand.push_back(BShape{r, zl});
        }
      // the class's instances of this batch together, as in the real launch; their
      // outputs go to each grid's scratch (the caller's T is not touched)
      std::vector<BInst> sub;
      std::vector<thermal_grid*> sg;
      std::vector<MGBDesc> smg;
      for (size_t i : members) {
        if (mgd) smg.push_back((*mgd)[i]);
        thermal_grid* g = gs[i];
        if (!g->stage_T) {
          if (cudaMalloc((void**)&g->stage_T, sizeof(double) * (size_t)g->n) != cudaSuccess) {
            cudaGetLastError();
            return th_fail(TH_ENOMEM, "staging allocation failed");
          }
        }
        BInst I = hi[i];
        I.T_in = nullptr;
        I.T_out = g->stage_T;
        sub.push_back(I);
        sg.push_back(g);
      }
      const std::vector<Ctl> c0(sub.size(), batch_ctl(opts, 0.0, 1, 3));
      float best = 1e30f;
      for (const BShape& c : cand) {
        for (BInst& I : sub) {
          I.rows = c.rows;
          I.zl = c.zc;
        }
        float ms = 0.f;
        TH_TRY(launch_batch(sub, sg, c0.data(), power_dtype, opts, k, 3, s, &ms, mgd ? &smg : nullptr));  // warm-up
        TH_TRY(launch_batch(sub, sg, c0.data(), power_dtype, opts, k, 3, s, &ms, mgd ? &smg : nullptr));
        if (ms < best) {
          best = ms;
          chosen = c;
        }
      }
      std::lock_guard<std::mutex> lk(g_rows_mu);
      g_rows[key] = chosen;
    }
    for (size_t i : members) {
      hi[i].rows = chosen.rows;
      hi[i].zl = chosen.zc;
    }
  }
  return TH_OK;
}

static th_status persistent(thermal_grid* const* grids, int n, const void* const* power, int power_dtype,
                            double* const* T, const thermal_solve_opts* opts, thermal_solve_stats* stats,
                            cudaStream_t s) {
  std::vector<BInst> hi(n);
  std::vector<thermal_grid*> gs(grids, grids + n);
  std::vector<std::vector<float>> c1s(n), c2s(n);
  std::vector<double> lmins(n), lmaxs(n);
  const int k = opts->precond == TH_PC_CHEB ? opts->cheb_degree : 1;
  const bool mg = opts->precond == TH_PC_MG;
  std::vector<MGBDesc> mgd(mg ? n : 0);
  for (int i = 0; i < n; ++i) {
    thermal_grid* g = grids[i];
    TH_TRY(grid_ensure_tab(g, 0.0, s));
    TH_TRY(grid_ensure_workspace(g, false, s));
    if (mg) TH_TRY(mg_batch_levels(g, &mgd[i], s));
    float inv_theta = 1.0f;
    if (opts->precond == TH_PC_CHEB)
      TH_TRY(solver_cheb_coeffs(g, 0.0, opts, c1s[i], c2s[i], &inv_theta, &lmins[i], &lmaxs[i], s));
    BInst& I = hi[i];
    I = BInst{};
    I.d = grid_dims(g);
    I.uni = g->uniform ? 1 : 0;
    I.rows = 1;
    I.zl = I.d.L;
    I.f32 = g->f32;
    I.f64 = g->f64;
    I.tab = g->tab;
    I.invd = g->invd32;
    I.P = power[i];
    I.T_in = opts->use_guess ? T[i] : nullptr;
    I.T_out = T[i];
    I.t_amb = g->t_amb;
    I.theta = g->theta[0];
    I.r = g->r32;
    I.dv = g->d32;
    I.p[0] = g->p32[0];
    I.p[1] = g->p32[1];
    I.mu = g->mu32;
    for (int q = 0; q < 3; ++q) I.zc[q] = g->zc32[q];
    I.inv_theta = inv_theta;
    I.ctl = g->ctl;
  }
  // per-instance Chebyshev coefficients
  DevArr<float> coef;
  TH_TRY(coef.alloc((size_t)2 * n * k));
  std::vector<float> hc((size_t)2 * n * k, 0.0f);
  for (int i = 0; i < n; ++i)
    for (int m = 0; m < k && opts->precond == TH_PC_CHEB; ++m) {
      hc[(size_t)(2 * i) * k + m] = c1s[i][m];
      hc[(size_t)(2 * i + 1) * k + m] = c2s[i][m];
    }
  TH_CUDA(cudaMemcpyAsync(coef.p, hc.data(), hc.size() * sizeof(float), cudaMemcpyHostToDevice, s));
  for (int i = 0; i < n; ++i) {
    hi[i].c1 = coef.p + (size_t)(2 * i) * k;
    hi[i].c2 = coef.p + (size_t)(2 * i + 1) * k;
  }
  TH_TRY(tune_rows(hi, gs, power_dtype, opts, k, s, mg ? &mgd : nullptr));
  std::vector<Ctl> c0(n, batch_ctl(opts, opts->tol_rel, opts->max_outer, opts->max_inner));
  float ms = 0.f;
  TH_TRY(launch_batch(hi, gs, c0.data(), power_dtype, opts, k,
                      std::max(1, opts->max_outer) * std::max(1, opts->max_inner), s, &ms, mg ? &mgd : nullptr));
  th_status first_bad = TH_OK;
  for (int i = 0; i < n; ++i) {
    Ctl h;
    TH_CUDA(cudaMemcpy(&h, grids[i]->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
    th_status st = (th_status)h.status;
    if (st == TH_OK && !(h.rel_res <= opts->tol_rel)) st = TH_ENOCONV;
    if (stats) {
      std::memset(&stats[i], 0, sizeof(stats[i]));
      stats[i].status = st;
      stats[i].outer_it = h.outer_it;
      stats[i].inner_it = h.it_total;
      stats[i].n_spmv = h.n_spmv + h.it_total * k + (long long)h.n_inits * (k - 1);
      stats[i].rel_res = h.rel_res;
      stats[i].t_solve_ms = ms;
      stats[i].lam_min = lmins[i];
      stats[i].lam_max = lmaxs[i];
      stats[i].tile_rows = hi[i].rows;
      stats[i].tile_layers = hi[i].zl;
    }
    if (st != TH_OK && first_bad == TH_OK) first_bad = st;
  }
  if (first_bad != TH_OK) return th_fail(first_bad, "at least one batched instance did not converge");
  return TH_OK;
}

extern "C" th_status thermal_solve_batched(thermal_grid* const* grids, int n, const void* const* power,
                                           int power_dtype, double* const* T, const thermal_solve_opts* opts,
                                           thermal_solve_stats* stats, void* stream) {
  try {
    th_clear_error();
    if (n < 0) return th_fail(TH_EINVAL, "n < 0");
    TH_TRY(validate_opts(opts));
    if (power_dtype != TH_F32 && power_dtype != TH_F64) return th_fail(TH_EINVAL, "power dtype");
    if (n == 0) return TH_OK;  // the arrays may be NULL when there is nothing to solve
    if (!grids || !power || !T) return th_fail(TH_EINVAL, "NULL argument");
    bool all_dev = true, v4 = true;
    for (int i = 0; i < n; ++i) {
      if (!grids[i] || !power[i] || !T[i]) return th_fail(TH_EINVAL, "instance %d has a NULL pointer", i);
      if (!grids[i]->geom) return th_fail(TH_ESTATE, "instance %d has no geometry", i);
      if (!(grids[i]->h > 0.0)) return th_fail(TH_EINVAL, "instance %d has h = 0 (G singular)", i);
      all_dev = all_dev && is_device_pointer(power[i]) && is_device_pointer(T[i]);
      v4 = v4 && grids[i]->nx % 4 == 0 && ((uintptr_t)power[i] % 16) == 0;
    }
    // every instance iterates in its grid's own work vectors and control block and
    // writes its own T: a grid or an output passed twice would be shared by two
    // instances of one launch, so both are rejected
    {
      std::vector<const void*> gs(grids, grids + n), ts(T, T + n);
      std::sort(gs.begin(), gs.end());
      std::sort(ts.begin(), ts.end());
      if (std::adjacent_find(gs.begin(), gs.end()) != gs.end())
        return th_fail(TH_EINVAL, "the same grid handle appears twice in the batch (one grid per instance)");
      if (std::adjacent_find(ts.begin(), ts.end()) != ts.end())
        return th_fail(TH_EINVAL, "the same output buffer T appears twice in the batch");
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the persistent kernel covers the mixed path with the Jacobi, Chebyshev, multigrid
    // and no preconditioner on grids with nx % 4 == 0; other combinations run the
    // instances one after another through the single-grid solver
    // multigrid in the persistent kernel: at most 8 layers and at least two levels
    // (max(nx, ny) > 8) on every instance
    bool mg_ok = true;
    for (int i = 0; i < n; ++i) mg_ok = mg_ok && grids[i]->L <= 8 && std::max(grids[i]->nx, grids[i]->ny) > 8;
    const bool fused = all_dev && v4 && opts->precision != TH_PREC_FP64 &&
                       (opts->precond == TH_PC_NONE || opts->precond == TH_PC_JACOBI || opts->precond == TH_PC_CHEB ||
                        (opts->precond == TH_PC_MG && mg_ok)) &&
                       opts->batched_mode == 0;
    if (fused) return persistent(grids, n, power, power_dtype, T, opts, stats, s);
    return sequential(grids, n, power, power_dtype, T, opts, stats, s);
  } catch (...) {
    return th_fail(TH_ECUDA, "unexpected C++ exception inside libthermal");
  }
}
