// Vectorised FP32 stencil kernels (used when nx % 4 == 0).
//
// Each thread owns 4 consecutive cells of one x-row (one 16-byte load per array)
// and walks a chunk of layers upwards: the z-1 / z+1 values and the face below
// stay in registers, so a cell costs one float4 load of the vector, its x/y
// neighbours come from the float4 itself, two scalar loads and the rows above /
// below (L1), and the face arrays are read once.  Faces outside the grid are
// stored as zeros, so boundary terms vanish without per-term branches (a missing
// neighbour's value is read as 0 and multiplied by a zero conductance).
//
// Launch: block (TH_BX, TH_BY4), grid (ceil(nx/(4*TH_BX)), ceil(ny/TH_BY4),
// ceil(L/zc)); requires nx % 4 == 0 and 16-byte aligned base pointers.
#pragma once

#include "common.cuh"
#include "dfloat.cuh"

#define TH_BY4 8

__device__ __forceinline__ float4 z4() { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, const float4& v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float4 ldc4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float4 ldc4(const __nv_bfloat16* p) {
  const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
  const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
  const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
  return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float cmp(const float4& v, int k) {
  return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

struct Walk4 {
  int x0, y, zs, ze;
  long long b0;  // index of (x0, y, 0)
  bool valid;
};

__device__ __forceinline__ Walk4 walk4_of(const Dims& d, int zc) {
  Walk4 w;
  w.x0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  w.y = blockIdx.y * blockDim.y + threadIdx.y;
  w.zs = blockIdx.z * zc;
  w.ze = min(w.zs + zc, d.L);
  w.valid = (w.x0 < d.nx) && (w.y < d.ny);
  w.b0 = (long long)w.x0 + (long long)d.nx * w.y;
  return w;
}

// Tiles (x block, y block, z chunk) of the z-walk, for kernels that walk them
// grid-stride (a grid of resident blocks pays a reduction's per-block tail once).
__device__ __forceinline__ int walk4_tiles(const Dims& d, int zc) {
  const int gbx = (d.nx + 4 * TH_BX - 1) / (4 * TH_BX), gby = (d.ny + TH_BY4 - 1) / TH_BY4;
  return gbx * gby * ((d.L + zc - 1) / zc);
}

__device__ __forceinline__ Walk4 walk4_tile(const Dims& d, int zc, int t) {
  const int gbx = (d.nx + 4 * TH_BX - 1) / (4 * TH_BX), gby = (d.ny + TH_BY4 - 1) / TH_BY4;
  const int bx = t % gbx, by = (t / gbx) % gby, bz = t / (gbx * gby);
  Walk4 w;
  w.x0 = 4 * (bx * TH_BX + threadIdx.x);
  w.y = by * TH_BY4 + threadIdx.y;
  w.zs = bz * zc;
  w.ze = min(w.zs + zc, d.L);
  w.valid = (w.x0 < d.nx) && (w.y < d.ny);
  w.b0 = (long long)w.x0 + (long long)d.nx * w.y;
  return w;
}

// Walks the layers of one 4-cell row segment.  V4(i) returns the operand at cells
// i..i+3 (float4), V1(j) at one cell.  For each layer z calls
// epi(i, z, v, acc, dg): v = operand, acc = (A v) and dg = A_ii for the 4 cells,
// accumulated in the order of stencil_row (s v, +x, -x, +y, -y, +z, -z).
__device__ __forceinline__ float4 f4s(float v) { return make_float4(v, v, v, v); }

// UNI: the grid has one conductivity per layer, so the face conductances come from
// the per-layer table (gxl, gyl, gzl) and are 0 on the domain boundary: no face
// arrays are read.  Otherwise they are read from the per-face arrays gx, gy, gz.
template <typename TC, bool UNI, typename F4, typename F1, typename E>
__device__ __forceinline__ void zwalk4(const Dims& d, const Walk4& w, const TC* __restrict__ gx,
                                       const TC* __restrict__ gy, const TC* __restrict__ gz, const LayerTab* tab,
                                       F4 V4, F1 V1, E epi) {
  const long long pxy = d.pxy;
  const bool hasL = w.x0 > 0, hasR = w.x0 + 4 < d.nx, hasD = w.y > 0, hasU = w.y + 1 < d.ny;
  float4 vb = z4(), gzb = z4();
  if (w.zs > 0) {
    vb = V4(w.b0 + (long long)(w.zs - 1) * pxy);
    gzb = UNI ? f4s(__ldg(&tab->gzl[w.zs - 1])) : ldc4(gz + w.b0 + (long long)(w.zs - 1) * pxy);
  }
  float4 vc = V4(w.b0 + (long long)w.zs * pxy);
  for (int z = w.zs; z < w.ze; ++z) {
    const long long i = w.b0 + (long long)z * pxy;
    const bool hasA = z + 1 < d.L;
    const float4 va = hasA ? V4(i + pxy) : z4();
    float4 gzv, gxv, gyv, gyd;
    float gxl;
    if (UNI) {
      const float cx = __ldg(&tab->gxl[z]), cy = __ldg(&tab->gyl[z]);
      gzv = f4s(hasA ? __ldg(&tab->gzl[z]) : 0.f);
      gxv = make_float4(cx, cx, cx, hasR ? cx : 0.f);
      gyv = f4s(hasU ? cy : 0.f);
      gyd = f4s(hasD ? cy : 0.f);
      gxl = hasL ? cx : 0.f;
    } else {
      gzv = hasA ? ldc4(gz + i) : z4();
      gxv = ldc4(gx + i);
      gyv = ldc4(gy + i);
      gyd = hasD ? ldc4(gy + i - d.nx) : z4();
      gxl = hasL ? ldc(gx + i - 1) : 0.f;
    }
    const float vl = hasL ? V1(i - 1) : 0.f;
    const float vr = hasR ? V1(i + 4) : 0.f;
    const float4 vu = hasU ? V4(i + d.nx) : z4();
    const float4 vd = hasD ? V4(i - d.nx) : z4();
    const float s = __ldg(&tab->s32[z]);
    float acc[4], dg[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float v = cmp(vc, k);
      const float right = (k == 3) ? vr : cmp(vc, k + 1);
      const float left = (k == 0) ? vl : cmp(vc, k - 1);
      const float gr = cmp(gxv, k);
      const float gl = (k == 0) ? gxl : cmp(gxv, k - 1);
      float a = s * v, g = s;
      a += gr * (v - right);        g += gr;
      a += gl * (v - left);         g += gl;
      a += cmp(gyv, k) * (v - cmp(vu, k));  g += cmp(gyv, k);
      a += cmp(gyd, k) * (v - cmp(vd, k));  g += cmp(gyd, k);
      a += cmp(gzv, k) * (v - cmp(va, k));  g += cmp(gzv, k);
      a += cmp(gzb, k) * (v - cmp(vb, k));  g += cmp(gzb, k);
      acc[k] = a;
      dg[k] = g;
    }
    epi(i, z, vc, acc, dg);
    vb = vc;
    vc = va;
    gzb = gzv;
  }
}

// One Chebyshev step (see k_cheb), vectorised.
template <typename TC, bool SCALED, bool LAST, bool UNI>
__global__ void __launch_bounds__(TH_BX* TH_BY4)
    k_cheb_v4(Dims d, int zc, Ctl* ctl, const TC* __restrict__ gx, const TC* __restrict__ gy,
              const TC* __restrict__ gz, const LayerTab* tab, const float* __restrict__ r,
              const float* __restrict__ zprev, const float* __restrict__ zcur, float* __restrict__ znext, float c1,
              float c2, double* partials, int stride, unsigned* counter) {
  if (ld_int(&ctl->done)) return;
  const Walk4 w = walk4_of(d, zc);
  float part[1] = {0.f};
  if (w.valid) {
    zwalk4<TC, UNI>(d, w, gx, gy, gz, tab, [&](long long i) { return ld4(zcur + i); },
               [&](long long j) { return zcur[j]; },
               [&](long long i, int, const float4& v, const float (&acc)[4], const float (&dg)[4]) {
                 const float4 rv = ld4(r + i);
                 const float4 zp = zprev ? ld4(zprev + i) : z4();
                 float o[4];
#pragma unroll
                 for (int k = 0; k < 4; ++k) {
                   const float vk = cmp(v, k);
                   float res = cmp(rv, k) - acc[k];
                   if (SCALED) res = res / dg[k];
                   o[k] = vk + c1 * (vk - cmp(zp, k)) + c2 * res;
                   if (LAST) part[0] += cmp(rv, k) * o[k];
                 }
                 st4(znext + i, make_float4(o[0], o[1], o[2], o[3]));
               });
  }
  if (!LAST) return;
  double tot[1];
  if (!grid_reduce<float, 1>(part, partials, stride, counter, tot)) return;
  ctl->rz_next = tot[0];
  ctl_set_beta(ctl);
}

// Search direction + stencil + p^T A p (see k_spmv_dot), vectorised.
template <bool UNI>
__global__ void __launch_bounds__(TH_BX* TH_BY4)
    k_spmv_dot_v4(Dims d, int zc, Ctl* ctl, const float* __restrict__ gx, const float* __restrict__ gy,
                  const float* __restrict__ gz, const LayerTab* tab, const float* __restrict__ z,
                  const float* __restrict__ p_old, float* __restrict__ p_new, float* __restrict__ mu,
                  double* partials, int stride, unsigned* counter) {
  if (ld_int(&ctl->done)) return;
  const int first = ld_int(&ctl->first);
  const float beta = first ? 0.f : ctl_beta<float>(ctl);
  float part[1] = {0.f};
  const int ntl = walk4_tiles(d, zc);
  for (int t = blockIdx.x; t < ntl; t += gridDim.x) {
    const Walk4 w = walk4_tile(d, zc, t);
    if (!w.valid) continue;
    auto P4 = [&](long long i) -> float4 {
      const float4 a = ld4(z + i);
      if (first) return a;
      const float4 b = ld4(p_old + i);
      return make_float4(a.x + beta * b.x, a.y + beta * b.y, a.z + beta * b.z, a.w + beta * b.w);
    };
    auto P1 = [&](long long j) -> float { return first ? z[j] : z[j] + beta * p_old[j]; };
    zwalk4<float, UNI>(d, w, gx, gy, gz, tab, P4, P1,
                  [&](long long i, int, const float4& v, const float (&acc)[4], const float (&)[4]) {
                    st4(p_new + i, v);
                    st4(mu + i, make_float4(acc[0], acc[1], acc[2], acc[3]));
#pragma unroll
                    for (int k = 0; k < 4; ++k) part[0] += cmp(v, k) * acc[k];
                  });
  }
  double tot[1];
  if (!grid_reduce<float, 1>(part, partials, stride, counter, tot)) return;
  fin_pap(ctl, tot[0]);
}

// y = A x, vectorised (FP32).
template <typename TC, bool UNI>
__global__ void __launch_bounds__(TH_BX* TH_BY4)
    k_apply_v4(Dims d, int zc, const TC* __restrict__ gx, const TC* __restrict__ gy, const TC* __restrict__ gz,
               const LayerTab* tab, const float* __restrict__ x, float* __restrict__ y) {
  const Walk4 w = walk4_of(d, zc);
  if (!w.valid) return;
  zwalk4<TC, UNI>(d, w, gx, gy, gz, tab, [&](long long i) { return ld4(x + i); }, [&](long long j) { return x[j]; },
             [&](long long i, int, const float4&, const float (&acc)[4], const float (&)[4]) {
               st4(y + i, make_float4(acc[0], acc[1], acc[2], acc[3]));
             });
}

// Vectorised k_update (element-wise; a thread handles groups of 4 consecutive
// cells, grid-stride, so that a grid of a few blocks per SM keeps the number of
// per-block partials of the reduction small).  TAB: a layer-uniform grid takes the
// inverse diagonal from the layer table's boundary-case entries (the row, y and z of
// a group from its index) instead of reading the per-cell array: 4 B/cell less.
template <bool INIT, int ZMODE, bool TAB>
static __global__ void __launch_bounds__(256)
    k_update_v4(long long n4, Ctl* ctl, float* __restrict__ x, const float* __restrict__ p, float* __restrict__ r,
                const float* __restrict__ mu, const float* __restrict__ invd, float* __restrict__ z, float zscale,
                int scaled, int rz_here, int scale_r, double* partials, int stride, unsigned* counter, Dims d,
                const LayerTab* tab) {
  if (!INIT && ld_int(&ctl->done)) return;
  if (INIT && ld_int(&ctl->outer_done)) return;
  const float alpha = INIT ? 0.f : ctl_alpha<float>(ctl);
  const float rs = (INIT && scale_r) ? __ldcg(&ctl->rscale_f) : 1.f;
  float v[2] = {0.f, 0.f};
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n4;
       q += (long long)gridDim.x * blockDim.x) {
    const long long i = 4 * q;
    float4 rv = ld4(r + i);
    float rr[4] = {rv.x, rv.y, rv.z, rv.w};
    if (INIT) {
      if (x) st4(x + i, z4());
      if (scale_r) {
#pragma unroll
        for (int k = 0; k < 4; ++k) rr[k] *= rs;
        st4(r + i, make_float4(rr[0], rr[1], rr[2], rr[3]));
      }
    } else {
      const float4 xv = ld4(x + i), pv = ld4(p + i), mv = ld4(mu + i);
      st4(x + i, make_float4(xv.x + alpha * pv.x, xv.y + alpha * pv.y, xv.z + alpha * pv.z, xv.w + alpha * pv.w));
      rr[0] -= alpha * mv.x; rr[1] -= alpha * mv.y; rr[2] -= alpha * mv.z; rr[3] -= alpha * mv.w;
      st4(r + i, make_float4(rr[0], rr[1], rr[2], rr[3]));
    }
    float zz[4] = {rr[0], rr[1], rr[2], rr[3]};
    if (ZMODE == 1 || (ZMODE == 2 && scaled)) {
      float4 iv;
      if (TAB) {  // row (y, z) and the group's place in it; nx % 4 == 0
        const unsigned n4r = (unsigned)d.nx >> 2;
        const unsigned row = (unsigned)q / n4r, x4 = (unsigned)q - row * n4r;
        const unsigned yy = row % (unsigned)d.ny, zz_ = row / (unsigned)d.ny;
        const int nyf = 3 * ((yy + 1 < (unsigned)d.ny) + (yy > 0));
        const float mid = __ldg(&tab->invd9[2 + nyf][zz_]), end = __ldg(&tab->invd9[1 + nyf][zz_]);
        iv = make_float4(x4 == 0 ? end : mid, mid, mid, x4 + 1 == n4r ? end : mid);
      } else {
        iv = __ldg(reinterpret_cast<const float4*>(invd + i));
      }
      zz[0] *= iv.x; zz[1] *= iv.y; zz[2] *= iv.z; zz[3] *= iv.w;
    }
    if (ZMODE == 2) {
#pragma unroll
      for (int k = 0; k < 4; ++k) zz[k] *= zscale;
    }
    if (ZMODE == 1 || ZMODE == 2) st4(z + i, make_float4(zz[0], zz[1], zz[2], zz[3]));
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[0] += rr[k] * rr[k];
      v[1] += rr[k] * zz[k];
    }
  }
  double tot[2];
  if (!grid_reduce<float, 2>(v, partials, stride, counter, tot)) return;
  fin_update(ctl, tot[0], tot[1], INIT, rz_here);
}

// power map values of 4 consecutive cells as double-floats
__device__ __forceinline__ void ldp4(const float* p, df (&o)[4]) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  o[0] = df_make(v.x, 0.f); o[1] = df_make(v.y, 0.f); o[2] = df_make(v.z, 0.f); o[3] = df_make(v.w, 0.f);
}
__device__ __forceinline__ void ldp4(const double* p, df (&o)[4]) {
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double v = __ldg(p + k);
    const float h = (float)v;
    o[k] = df_make(h, (float)(v - (double)h));
  }
}

// The double-float refinement residual (see k_residual_df) on a layer-uniform
// grid, vectorised: per cell r = P + cdt (theta_n - theta) - sink theta - flux with
// flux = gx (2 theta - theta_r - theta_l) + gy (2 theta - theta_u - theta_d)
//      + gza (theta - theta_above) + gzb (theta - theta_below),
// an absent neighbour taking the cell's own value (its difference is exactly 0).
// The seven differences are normalised double-floats; the sums, products and the
// accumulation use the unnormalised forms (about 165 FP32 operations per cell
// instead of 230).  The difference form matters: its products are
// g (theta - theta_f), small for a smooth field, whereas the expanded form's
// D theta and g theta_f are large and cancel, leaving an absolute error of order
// 2^-47 D |theta| that stalls the refinement near 1e-10 on stacks with a Cu
// spreader.  Likewise an unnormalised difference whose high parts cancel keeps its
// whole value in the low part, and the next sum then rounds it relative to |theta|
// rather than to the difference.
//
// ZI >= 0 also starts the inner solve on the unscaled r (what k_update_v4<true, ZI>
// does after it): x = 0, z = r (ZI 0), D^-1 r (1) or zs (D^-1) r (2, D^-1 when
// `scaled`), and r^T z; the last block then makes the inner solve's start decision
// unless the system has converged, and the correction is applied with scale 1.
struct ResidInit {
  float* x;
  float* z;
  float zs;
  int scaled, rz_here;
};

// UNI: layer-uniform grid, face conductances (hi, lo) from the per-layer table.
// Otherwise the per-face arrays: fh = FP32 high parts, fl = low parts g - (float)g
// (zero on the domain boundary), six face products per cell.
template <typename TP, int ZI, bool UNI>
// two blocks per SM (128 registers): the layer-table form on paired instructions
// spills at three (80 registers) and measured slower there (76.1 vs 72.3 us)
__global__ void __launch_bounds__(TH_BX* TH_BY4, 2)
    k_residual_df_v4(Dims d, int zc, Ctl* ctl, const LayerTab* tab, Faces32 fh, Faces32 fl,
                     const float* __restrict__ th_hi, const float* __restrict__ th_lo, const TP* const* ptab,
                     const float* __restrict__ thn_hi, const float* __restrict__ thn_lo, float* __restrict__ r,
                     int count_outer, ResidInit ri, double* partials, int stride, unsigned* counter) {
  if (ld_int(&ctl->outer_done)) return;
  const TP* P = ptab[ld_int(&ctl->map_idx)];
  float v[3] = {0.f, 0.f, 0.f};
  const int ntl = walk4_tiles(d, zc);
  for (int t = blockIdx.x; t < ntl; t += gridDim.x) {
    const Walk4 w = walk4_tile(d, zc, t);
    if (!w.valid) continue;
    const long long pxy = d.pxy;
    const bool hasL = w.x0 > 0, hasR = w.x0 + 4 < d.nx, hasD = w.y > 0, hasU = w.y + 1 < d.ny;
    float4 hb = z4(), lb = z4();
    float4 gbh = z4(), gbl = z4();  // per-face grids: the faces below the current layer
    if (w.zs > 0) {
      hb = ld4(th_hi + w.b0 + (long long)(w.zs - 1) * pxy);
      lb = ld4(th_lo + w.b0 + (long long)(w.zs - 1) * pxy);
      if (!UNI) {
        gbh = ldc4(fh.gz + w.b0 + (long long)(w.zs - 1) * pxy);
        gbl = ldc4(fl.gz + w.b0 + (long long)(w.zs - 1) * pxy);
      }
    }
    float4 hc = ld4(th_hi + w.b0 + (long long)w.zs * pxy), lc = ld4(th_lo + w.b0 + (long long)w.zs * pxy);
    for (int z = w.zs; z < w.ze; ++z) {
      const long long i = w.b0 + (long long)z * pxy;
      const bool hasA = z + 1 < d.L, hasB = z > 0;
      const float4 ha = hasA ? ld4(th_hi + i + pxy) : hc, la = hasA ? ld4(th_lo + i + pxy) : lc;
      const float4 hu = hasU ? ld4(th_hi + i + d.nx) : hc, lu = hasU ? ld4(th_lo + i + d.nx) : lc;
      const float4 hd = hasD ? ld4(th_hi + i - d.nx) : hc, ld_ = hasD ? ld4(th_lo + i - d.nx) : lc;
      const float hl1 = hasL ? th_hi[i - 1] : hc.x, ll1 = hasL ? th_lo[i - 1] : lc.x;
      const float hr1 = hasR ? th_hi[i + 4] : hc.w, lr1 = hasR ? th_lo[i + 4] : lc.w;
      const float4 hbz = hasB ? hb : hc, lbz = hasB ? lb : lc;
      df pv[4];
      ldp4(P + i, pv);
      float4 nh = z4(), nl = z4();
      if (thn_hi) {
        nh = ld4(thn_hi + i);
        nl = ld4(thn_lo + i);
      }
      const df sk = df_make(__ldg(&tab->sink_hi[z]), __ldg(&tab->sink_lo[z]));
      const df cd = df_make(__ldg(&tab->cdt_hi[z]), __ldg(&tab->cdt_lo[z]));
      df gx, gy, ga, gb;  // layer table
      float4 gxh, gxl_, gyh, gyl_, gdh, gdl, gah, gal;  // per-face arrays
      float gLh = 0.f, gLl = 0.f;
      if (UNI) {
        gx = df_make(__ldg(&tab->gxl_hi[z]), __ldg(&tab->gxl_lo[z]));
        gy = df_make(__ldg(&tab->gyl_hi[z]), __ldg(&tab->gyl_lo[z]));
        ga = df_make(__ldg(&tab->gzl_hi[z]), __ldg(&tab->gzl_lo[z]));
        gb = hasB ? df_make(__ldg(&tab->gzl_hi[z - 1]), __ldg(&tab->gzl_lo[z - 1])) : df_make(0.f, 0.f);
      } else {
        gxh = ldc4(fh.gx + i);
        gxl_ = ldc4(fl.gx + i);
        gyh = ldc4(fh.gy + i);
        gyl_ = ldc4(fl.gy + i);
        gdh = hasD ? ldc4(fh.gy + i - d.nx) : z4();
        gdl = hasD ? ldc4(fl.gy + i - d.nx) : z4();
        gah = hasA ? ldc4(fh.gz + i) : z4();
        gal = hasA ? ldc4(fl.gz + i) : z4();
        if (hasL) {
          gLh = ldc(fh.gx + i - 1);
          gLl = ldc(fl.gx + i - 1);
        }
      }
      float o[4];
      if constexpr (UNI) {
        // cells (0, 1) and (2, 3) in the two lanes of the paired instructions; per
        // cell: the power, the sink and transient terms, then the normalised
        // neighbour differences with unnormalised sums, products and accumulation
        // (as in the per-face form below)
        float bhv[4];
        const df2 gx2 = df2_of(gx, gx), gy2 = df2_of(gy, gy), ga2 = df2_of(ga, ga), gb2 = df2_of(gb, gb);
        const df2 sk2 = df2_of(sk, sk), cd2 = df2_of(cd, cd);
#pragma unroll
        for (int pr = 0; pr < 2; ++pr) {
          const int k0 = 2 * pr, k1 = 2 * pr + 1;
          auto pair = [&](const float4& h, const float4& l) {
            return df2_make(make_float2(cmp(h, k0), cmp(h, k1)), make_float2(cmp(l, k0), cmp(l, k1)));
          };
          const df2 t = pair(hc, lc);
          const df2 tr = pr ? df2_make(make_float2(hc.w, hr1), make_float2(lc.w, lr1))
                            : df2_make(make_float2(hc.y, hc.z), make_float2(lc.y, lc.z));
          const df2 tl = pr ? df2_make(make_float2(hc.y, hc.z), make_float2(lc.y, lc.z))
                            : df2_make(make_float2(hl1, hc.x), make_float2(ll1, lc.x));
          df2 acc = df2_of(pv[k0], pv[k1]);
          if (sk.hi != 0.f) acc = ldf2_sub(acc, ldf2_mul(sk2, t));
          float bh0 = pv[k0].hi, bh1 = pv[k1].hi;
          if (thn_hi) {
            acc = ldf2_add(acc, ldf2_mul(cd2, df2_sub(pair(nh, nl), t)));
            bh0 = __fmaf_rn(cd.hi, cmp(nh, k0), bh0);
            bh1 = __fmaf_rn(cd.hi, cmp(nh, k1), bh1);
          }
          const df2 dx = ldf2_add(df2_sub(t, tr), df2_sub(t, tl));
          const df2 dy = ldf2_add(df2_sub(t, pair(hu, lu)), df2_sub(t, pair(hd, ld_)));
          acc = ldf2_sub(acc, ldf2_mul(gx2, dx));
          acc = ldf2_sub(acc, ldf2_mul(gy2, dy));
          acc = ldf2_sub(acc, ldf2_mul(ga2, df2_sub(t, pair(ha, la))));
          acc = ldf2_sub(acc, ldf2_mul(gb2, df2_sub(t, pair(hbz, lbz))));
          o[k0] = acc.hi.x + acc.lo.x;
          o[k1] = acc.hi.y + acc.lo.y;
          bhv[k0] = bh0;
          bhv[k1] = bh1;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          v[0] += o[k] * o[k];
          v[1] += bhv[k] * bhv[k];
        }
      } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const df t = df_make(cmp(hc, k), cmp(lc, k));
        const df tr = (k == 3) ? df_make(hr1, lr1) : df_make(cmp(hc, k + 1), cmp(lc, k + 1));
        const df tl = (k == 0) ? df_make(hl1, ll1) : df_make(cmp(hc, k - 1), cmp(lc, k - 1));
        const df tu = df_make(cmp(hu, k), cmp(lu, k)), td = df_make(cmp(hd, k), cmp(ld_, k));
        const df ta = df_make(cmp(ha, k), cmp(la, k)), tb = df_make(cmp(hbz, k), cmp(lbz, k));
        df acc = pv[k];
        if (sk.hi != 0.f) acc = ldf_sub(acc, ldf_mul(sk, t));  // the sink is on the top layer only
        float bh = pv[k].hi;  // ||b|| needs FP32 accuracy only
        if (thn_hi) {
          const df tn = df_make(cmp(nh, k), cmp(nl, k));
          acc = ldf_add(acc, ldf_mul(cd, df_sub(tn, t)));
          bh = __fmaf_rn(cd.hi, tn.hi, bh);
        }
        // the neighbour differences are normalised (their high parts often cancel
        // exactly); the sums, products and the accumulation run unnormalised
        const df gR = df_make(cmp(gxh, k), cmp(gxl_, k));
        const df gL = (k == 0) ? df_make(gLh, gLl) : df_make(cmp(gxh, k - 1), cmp(gxl_, k - 1));
        acc = ldf_sub(acc, ldf_mul(gR, df_sub(t, tr)));
        acc = ldf_sub(acc, ldf_mul(gL, df_sub(t, tl)));
        acc = ldf_sub(acc, ldf_mul(df_make(cmp(gyh, k), cmp(gyl_, k)), df_sub(t, tu)));
        acc = ldf_sub(acc, ldf_mul(df_make(cmp(gdh, k), cmp(gdl, k)), df_sub(t, td)));
        acc = ldf_sub(acc, ldf_mul(df_make(cmp(gah, k), cmp(gal, k)), df_sub(t, ta)));
        acc = ldf_sub(acc, ldf_mul(df_make(cmp(gbh, k), cmp(gbl, k)), df_sub(t, tb)));
        o[k] = acc.hi + acc.lo;
        v[0] += o[k] * o[k];
        v[1] += bh * bh;
      }
      }
      st4(r + i, make_float4(o[0], o[1], o[2], o[3]));
      if (ZI >= 0) {
        st4(ri.x + i, z4());
        float zz[4] = {o[0], o[1], o[2], o[3]};
        if (ZI == 1 || (ZI == 2 && ri.scaled)) {  // inverse diagonal from the boundary-case table
          const int nyf = 3 * ((int)hasU + (int)hasD);
          const float mid = __ldg(&tab->invd9[2 + nyf][z]), end = __ldg(&tab->invd9[1 + nyf][z]);
          zz[0] *= hasL ? mid : end;
          zz[1] *= mid;
          zz[2] *= mid;
          zz[3] *= hasR ? mid : end;
        }
        if (ZI == 2) {
#pragma unroll
          for (int k = 0; k < 4; ++k) zz[k] *= ri.zs;
        }
        if (ZI >= 1) st4(ri.z + i, make_float4(zz[0], zz[1], zz[2], zz[3]));
#pragma unroll
        for (int k = 0; k < 4; ++k) v[2] += o[k] * zz[k];
      }
      hb = hc; lb = lc;
      hc = ha; lc = la;
      if (!UNI) {
        gbh = gah;
        gbl = gal;
      }
    }
  }
  double tot[3];
  if (!grid_reduce<float, 3>(v, partials, stride, counter, tot)) return;
  fin_residual(ctl, tot[0], tot[1], 0, count_outer);
  if (ZI >= 0) {
    ctl->rnorm_hi = 1.f;  // the inner solve runs on the unscaled r
    ctl->rnorm_lo = 0.f;
    if (!ctl->outer_done) fin_update(ctl, tot[0], tot[2], true, ri.rz_here);
  }
}

// Element-wise double-float kernels of the mixed path, 4 cells per thread (n % 4 == 0,
// 16-byte aligned arrays); the loop scalars are read once per thread.

// theta += ||r|| d (see k_theta_axpy_df).
static __global__ void __launch_bounds__(256)
    k_theta_axpy_df_v4(long long n4, const Ctl* ctl, float* __restrict__ th_hi, float* __restrict__ th_lo,
                       const float* __restrict__ d) {
  if (ld_int(&ctl->outer_done)) return;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n4) return;
  const long long i = 4 * q;
  const df rn = df_make(__ldcg(&ctl->rnorm_hi), __ldcg(&ctl->rnorm_lo));
  const float4 h = ld4(th_hi + i), l = ld4(th_lo + i), dv = ld4(d + i);
  float oh[4], ol[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const df t = df_add(df_make(cmp(h, k), cmp(l, k)), df_mul_f(rn, cmp(dv, k)));
    oh[k] = t.hi;
    ol[k] = t.lo;
  }
  st4(th_hi + i, make_float4(oh[0], oh[1], oh[2], oh[3]));
  st4(th_lo + i, make_float4(ol[0], ol[1], ol[2], ol[3]));
}

// Start of a step with the extrapolated guess (see k_step_extrap_df).
static __global__ void __launch_bounds__(256)
    k_step_extrap_df_v4(long long n4, float* th_hi, float* th_lo, float* thm_hi, float* thm_lo) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n4) return;
  const long long i = 4 * q;
  const float4 ch = ld4(th_hi + i), cl = ld4(th_lo + i), ph = ld4(thm_hi + i), pl = ld4(thm_lo + i);
  float gh[4], gl[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const df cur = df_make(cmp(ch, k), cmp(cl, k));
    const df g = df_sub(df_add(cur, cur), df_make(cmp(ph, k), cmp(pl, k)));
    gh[k] = g.hi;
    gl[k] = g.lo;
  }
  st4(thm_hi + i, ch);
  st4(thm_lo + i, cl);
  st4(th_hi + i, make_float4(gh[0], gh[1], gh[2], gh[3]));
  st4(th_lo + i, make_float4(gl[0], gl[1], gl[2], gl[3]));
}

// Start of a time step with an extrapolated guess (double-float, 4 cells per
// thread): theta <- the polynomial extrapolation of order q through theta_n and the
// history, and the history moves back by one step (thm <- theta_n, thm2 <- thm,
// thm3 <- thm2).  q = min(ORD, steps taken, steps taken since the power map last
// switched): the history before a switch follows another forcing, and extrapolating
// across the switch gives a worse start than a lower order (measured with the oracle
// on the 100-step workload shape).
//   q = 1: 2 t_n - t_{n-1};  q = 2: 3 t_n - 3 t_{n-1} + t_{n-2};
//   q = 3: 4 t_n - 6 t_{n-1} + 4 t_{n-2} - t_{n-3}.
template <int ORD>
static __global__ void __launch_bounds__(256)
    k_step_extrapq_df_v4(long long n4, const Ctl* ctl, float* th_hi, float* th_lo, float* thm_hi, float* thm_lo,
                         float* thm2_hi, float* thm2_lo, float* thm3_hi, float* thm3_lo) {
  const long long q4 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q4 >= n4) return;
  const int step = ld_int(&ctl->step);
  const int spm = ld_int(&ctl->steps_per_map), nmaps = ld_int(&ctl->n_maps);
  const int since = (nmaps > 1 && spm > 0) ? step % spm : step;
  const int q = min(ORD, min(step, since));
  const long long i = 4 * q4;
  const float4 ch = ld4(th_hi + i), cl = ld4(th_lo + i), ph = ld4(thm_hi + i), pl = ld4(thm_lo + i);
  const float4 qh = ld4(thm2_hi + i), ql = ld4(thm2_lo + i);
  float4 rh = z4(), rl = z4();
  if (ORD >= 3) {
    rh = ld4(thm3_hi + i);
    rl = ld4(thm3_lo + i);
  }
  float gh[4], gl[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const df cur = df_make(cmp(ch, k), cmp(cl, k));
    const df prev = df_make(cmp(ph, k), cmp(pl, k));
    df g = cur;
    if (q == 1) g = df_sub(df_add(cur, cur), prev);
    if (q == 2) g = df_add(df_mul_f(df_sub(cur, prev), 3.0f), df_make(cmp(qh, k), cmp(ql, k)));
    if (ORD >= 3 && q == 3) {
      // 4 (t_n - t_{n-1}) - 2 (t_{n-1} - t_{n-2}) + (t_{n-2} - t_{n-3}) + t_{n-2}
      const df p2 = df_make(cmp(qh, k), cmp(ql, k)), p3 = df_make(cmp(rh, k), cmp(rl, k));
      g = df_add(df_sub(df_mul_f(df_sub(cur, prev), 4.0f), df_mul_f(df_sub(prev, p2), 2.0f)),
                 df_add(df_sub(p2, p3), p2));
    }
    gh[k] = g.hi;
    gl[k] = g.lo;
  }
  if (ORD >= 3) {
    st4(thm3_hi + i, qh);
    st4(thm3_lo + i, ql);
  }
  st4(thm2_hi + i, ph);
  st4(thm2_lo + i, pl);
  st4(thm_hi + i, ch);
  st4(thm_lo + i, cl);
  st4(th_hi + i, make_float4(gh[0], gh[1], gh[2], gh[3]));
  st4(th_lo + i, make_float4(gl[0], gl[1], gl[2], gl[3]));
}
