// DDE-extended de-gridding and gridding (Section 2.1, the paragraph after Eq. 1), for
// sm_103a.  Included at the end of nufft.cu (it uses that file's Kaiser-Bessel taps,
// grid layout and block reductions).
//
// Row m of G_l is the Kaiser-Bessel kernel convolved with the visibility's compact
// Fourier-domain DDE kernel K_m ((2R + 1)^2 complex, R <= 4):
//   g_m[k] = sum_j K_m[j] phi(t_r - (k_r - j_r)) phi(t_c - (k_c - j_c)),
// a footprint of F x F cells, F = 7 + 2R (15 x 15 for 9 x 9 kernels), from cell
// (k0_r - R, k0_c - R), k0 the first Kaiser-Bessel tap.  In footprint coordinates
// (row r, column c; kernel index j1, j2 in [0, 2R]; taps a = r - j1, b = c - j2):
//   de-gridding  u_m = sum_{j1,j2} K[j1][j2] sum_a w_r[a] sum_b w_c[b] x[j1 + a][j2 + b]
//   gridding     x[r][c] += sum_b w_c[b] sum_a w_r[a] conj(K[r - a][c - b]) v_m
// Both are separable passes through per-warp shared-memory scratch: one warp works on
// one visibility at a time (its lanes split the footprint cells, the row and column
// passes and the kernel coefficients), so the kernel coefficients and the grid window
// are read coalesced once per visibility.
//
// Gridding keeps the scheme of k_grid: one CTA per (grid tile, channel) owns the tile's
// cells in shared memory and adds, in 32-bit fixed point with integer atomics (order-
// independent, so bitwise deterministic), every footprint cell that falls in the tile.
// Visibilities are bucketed by the tile of their first tap, and a footprint (F <= 15 <
// tile side) reaches only the 3 x 3 neighbouring tiles, so a CTA scans those buckets,
// keeps (by warp ballot) the visibilities whose footprint meets its tile, and processes
// them one by one.  The scale S = 2^e of a tile satisfies n_c m S < 2^30 with n_c the
// largest number of extended footprints covering one of its cells (counted once per
// kernel set, MODE 1) and m = max over the contributing visibilities of
// max(|Re v|, |Im v|) * sum_j (|Re K_j| + |Im K_j|), a bound of every tap value
// |Re|, |Im| of conj(g_m[k]) v_m (Kaiser-Bessel weights are at most 1).

namespace fhs {

constexpr int kDdeThreads = 256;
constexpr int kDdeWarps = kDdeThreads / 32;

// Per-warp scratch; WIN: with the grid window (de-gridding only).
template <int R, bool WIN>
struct DdeScratch {
  static constexpr int SD = 2 * R + 1;
  static constexpr int F = kTaps + 2 * R;
  float2 win[WIN ? F * F : 1];   // de-gridding: the grid window of the footprint
  float2 mid[F * SD];            // de-gridding: column pass; gridding: H[r][j2]
  float2 ker[SD * SD];           // de-gridding: K; gridding: conj(K) v S
  float w[2 * kTaps];            // row weights, then column weights
};

// Row and column Kaiser-Bessel weights of (xr, xc) into s.w (lanes 0..13).
template <class Scr>
__device__ __forceinline__ void dde_weights(Scr& s, float xr, float xc, int lane) {
  if (lane < kTaps) s.w[lane] = kb_tap(lane, xr);
  else if (lane < 2 * kTaps) s.w[lane] = kb_tap(lane - kTaps, xc);
}

// u_m of one visibility by the whole warp (same value returned on every lane).
template <int R>
__device__ __forceinline__ float2 dde_degrid_one(const float2* __restrict__ gl, float2 uvm,
                                                 const float2* __restrict__ Km, const VisGeom& vg,
                                                 DdeScratch<R, true>& s, int lane) {
  constexpr int SD = 2 * R + 1, F = kTaps + 2 * R;
  float xr, xc;
  const int kr = kb_first(uvm.y, vg.tc.hi_r, vg.tc.lo_r, xr);
  const int kc = kb_first(uvm.x, vg.tc.hi_c, vg.tc.lo_c, xc);
  dde_weights(s, xr, xc, lane);
  for (int k = lane; k < SD * SD; k += 32) s.ker[k] = Km[k];
  for (int k = lane; k < F * F; k += 32) {
    const int r = k / F, c = k - r * F;
    const int row = phys_row2(wrap1(kr - R + r, vg), vg);
    s.win[k] = gl[(size_t)row * vg.K2 + wrap2(kc - R + c, vg)];
  }
  __syncwarp();
  float wc[kTaps], wr[kTaps];
#pragma unroll
  for (int b = 0; b < kTaps; ++b) {
    wr[b] = s.w[b];
    wc[b] = s.w[kTaps + b];
  }
  // column pass: mid[r][j2] = sum_b w_c[b] win[r][j2 + b]
  for (int k = lane; k < F * SD; k += 32) {
    const int r = k / SD, j2 = k - r * SD;
    const float2* p = s.win + r * F + j2;
    float2 a = make_float2(0.f, 0.f);
#pragma unroll
    for (int b = 0; b < kTaps; ++b) {
      a.x = fmaf(wc[b], p[b].x, a.x);
      a.y = fmaf(wc[b], p[b].y, a.y);
    }
    s.mid[k] = a;
  }
  __syncwarp();
  // row pass and the kernel: u = sum_j K[j] sum_a w_r[a] mid[j1 + a][j2]
  float2 u = make_float2(0.f, 0.f);
  for (int k = lane; k < SD * SD; k += 32) {
    const int j1 = k / SD, j2 = k - j1 * SD;
    const float2* p = s.mid + j1 * SD + j2;
    float2 I = make_float2(0.f, 0.f);
#pragma unroll
    for (int a = 0; a < kTaps; ++a) {
      I.x = fmaf(wr[a], p[a * SD].x, I.x);
      I.y = fmaf(wr[a], p[a * SD].y, I.y);
    }
    const float2 K = s.ker[k];
    u.x = fmaf(K.x, I.x, fmaf(-K.y, I.y, u.x));
    u.y = fmaf(K.x, I.y, fmaf(K.y, I.x, u.y));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    u.x += __shfl_xor_sync(0xffffffffu, u.x, o);
    u.y += __shfl_xor_sync(0xffffffffu, u.y, o);
  }
  __syncwarp();                         // the scratch is reused by the next visibility
  return u;
}

// MODE 0: out[i] = u_i.  MODE 1: the PDFB data step of k_degrid_pdfb (z = v + 2u - u_prev,
// d = z - y, u_prev <- u, per-block FP64 partial sums).  CTA = 256 consecutive
// visibilities of channel blockIdx.y; warp w computes those of lanes 32 w .. 32 w + 31
// one by one, and lane t keeps the t-th result for the per-visibility epilogue.
template <int R, int MODE>
__global__ void __launch_bounds__(kDdeThreads) k_degrid_dde(const float2* __restrict__ grid,
                                                            const float2* __restrict__ uv,
                                                            const float2* __restrict__ kern,
                                                            const int32_t* __restrict__ kidx,
                                                            const int64_t* __restrict__ vis_off, VisGeom vg,
                                                            float2* __restrict__ out, const float2* __restrict__ y,
                                                            const float2* __restrict__ v, float2* __restrict__ u_prev,
                                                            const uint8_t* __restrict__ blk, int B,
                                                            double* __restrict__ partials, int nparts) {
  constexpr int SD = 2 * R + 1;
  __shared__ DdeScratch<R, true> scr[kDdeWarps];
  __shared__ double sred[kDdeWarps * 2 * kMaxB];
  const int l = blockIdx.y, lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t end = vis_off[l + 1];
  const int64_t wbase = vis_off[l] + (int64_t)blockIdx.x * kDdeThreads + wid * 32;
  const float2* gl = grid + (size_t)l * vg.K1 * vg.K2;
  float2 mine = make_float2(0.f, 0.f);
  for (int t = 0; t < 32; ++t) {
    const int64_t i = wbase + t;
    if (i >= end) break;                               // warp-uniform
    const float2 u = dde_degrid_one<R>(gl, uv[i], kern + (size_t)kidx[i] * SD * SD, vg, scr[wid], lane);
    if (lane == t) mine = u;
  }
  const int64_t i = wbase + lane;
  const bool valid = i < end;
  if (MODE == 0) {
    if (valid) out[i] = mine;
    return;
  }
  double v0 = 0.0, v1 = 0.0;
  int b = 0;
  if (valid) {
    const float2 yy = y[i], vv = v[i], up = u_prev[i];
    const float2 z = make_float2(vv.x + 2.f * mine.x - up.x, vv.y + 2.f * mine.y - up.y);
    const float2 d = make_float2(z.x - yy.x, z.y - yy.y);
    out[i] = d;
    u_prev[i] = mine;
    b = blk[i];
    v0 = (double)d.x * d.x + (double)d.y * d.y;
    const double rx = (double)yy.x - mine.x, ry = (double)yy.y - mine.y;
    v1 = rx * rx + ry * ry;
  }
  block_partials<kDdeWarps>(v0, v1, b, valid, B, sred, partials + ((size_t)l * nparts + blockIdx.x) * 2 * B);
}

// Local start (mod K) of a footprint that starts at absolute cell k, relative to tile
// start t0: cells (d + r) mod K < T of the footprint lie in the tile.
__device__ __forceinline__ int dde_local(int k, int t0, int K, int pw) {
  const int d = k - t0;
  return pw ? (d & (K - 1)) : ((d % K) + K) % K;
}

// Whether a footprint of F cells starting at local offset d (mod K) meets [0, T).
__device__ __forceinline__ bool dde_meets(int d, int F, int T, int K) { return d < T || d + F - 1 >= K; }

// Adds the footprint cells of one visibility that lie in the tile (MODE 0: fixed-point
// values of conj(g) v S, with vS = v S; MODE 1: one count per cell), by the whole warp.
template <int R, int MODE>
__device__ __forceinline__ void dde_grid_one(int* are, int* aim, int TP, int T, int dr, int dc, float xr, float xc,
                                             float2 vS, const float2* __restrict__ Km, const VisGeom& vg,
                                             DdeScratch<R, false>& s, int lane) {
  constexpr int SD = 2 * R + 1, F = kTaps + 2 * R;
  if (MODE == 1) {
    for (int k = lane; k < F * F; k += 32) {
      const int r = k / F, c = k - r * F;
      const int lr = wrap1(dr + r, vg), lc = wrap2(dc + c, vg);
      if (lr < T && lc < T) atomicAdd(are + lr * TP + lc, 1);
    }
    return;
  }
  dde_weights(s, xr, xc, lane);
  for (int k = lane; k < SD * SD; k += 32) {
    const float2 K = Km[k];
    s.ker[k] = make_float2(fmaf(K.x, vS.x, K.y * vS.y), fmaf(K.x, vS.y, -K.y * vS.x));   // conj(K) v S
  }
  __syncwarp();
  float wc[kTaps], wr[kTaps];
#pragma unroll
  for (int b = 0; b < kTaps; ++b) {
    wr[b] = s.w[b];
    wc[b] = s.w[kTaps + b];
  }
  // row pass: H[r][j2] = sum_a w_r[a] Z[r - a][j2]
  for (int k = lane; k < F * SD; k += 32) {
    const int r = k / SD, j2 = k - r * SD;
    float2 h = make_float2(0.f, 0.f);
#pragma unroll
    for (int a = 0; a < kTaps; ++a) {
      const int j1 = r - a;
      if (j1 >= 0 && j1 < SD) {
        const float2 z = s.ker[j1 * SD + j2];
        h.x = fmaf(wr[a], z.x, h.x);
        h.y = fmaf(wr[a], z.y, h.y);
      }
    }
    s.mid[k] = h;
  }
  __syncwarp();
  // column pass and the tile's cells: x[r][c] = sum_b w_c[b] H[r][c - b]
  for (int k = lane; k < F * F; k += 32) {
    const int r = k / F, c = k - r * F;
    const int lr = wrap1(dr + r, vg), lc = wrap2(dc + c, vg);
    if (lr >= T || lc >= T) continue;
    float2 x = make_float2(0.f, 0.f);
#pragma unroll
    for (int b = 0; b < kTaps; ++b) {
      const int j2 = c - b;
      if (j2 >= 0 && j2 < SD) {
        const float2 h = s.mid[r * SD + j2];
        x.x = fmaf(wc[b], h.x, x.x);
        x.y = fmaf(wc[b], h.y, x.y);
      }
    }
    atomicAdd(are + lr * TP + lc, __float2int_rn(x.x));
    atomicAdd(aim + lr * TP + lc, __float2int_rn(x.y));
  }
  __syncwarp();
}

// Source bucket s (0..8) of tile (tr, tc): the tile at offset (s / 3 - 1, s % 3 - 1),
// or -1 when it repeats an earlier one (fewer than 3 tiles along an axis).
__device__ __forceinline__ int dde_source(int s, int tr, int tc, int ntr, int ntc) {
  const int sr = (tr + s / 3 - 1 + ntr) % ntr, sc = (tc + s % 3 - 1 + ntc) % ntc;
  for (int e = 0; e < s; ++e) {
    const int er = (tr + e / 3 - 1 + ntr) % ntr, ec = (tc + e % 3 - 1 + ntc) % ntc;
    if (er == sr && ec == sc) return -1;
  }
  return sr * ntc + sc;
}

// MODE 0: grid the (block-scaled) values into tile blockIdx.x of channel blockIdx.y and
// store it (v_write, when set, receives the scaled values of the tile's own
// visibilities); MODE 1: store the tile's largest footprint count of a cell in
// ncmax[l][tile].
template <int R, int MODE>
__global__ void __launch_bounds__(kDdeThreads) k_grid_dde(const float2* __restrict__ vals,
                                                          const float* __restrict__ blk_scale,
                                                          float2* __restrict__ v_write, const float2* __restrict__ uv,
                                                          const uint8_t* __restrict__ blk,
                                                          const float2* __restrict__ kern,
                                                          const int32_t* __restrict__ kidx,
                                                          const float* __restrict__ kl1,
                                                          const int32_t* __restrict__ tile_off,
                                                          const int64_t* __restrict__ vis_off,
                                                          float2* __restrict__ grid, int* __restrict__ ncmax,
                                                          VisGeom vg, int T, int ntr, int ntc, int B) {
  constexpr int SD = 2 * R + 1, F = kTaps + 2 * R;
  extern __shared__ __align__(16) int dde_acc[];
  __shared__ DdeScratch<R, false> scr[kDdeWarps];
  __shared__ float sred[kDdeWarps];
  __shared__ int sredi[kDdeWarps];
  const int TP = grid_row_stride(T);
  int* are = dde_acc;
  int* aim = are + T * TP;
  const int l = blockIdx.y, tau = blockIdx.x, tr = tau / ntc, tc = tau % ntc;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  {
    int4* z4 = reinterpret_cast<int4*>(dde_acc);
    const int n4 = (MODE == 1 ? T * TP : 2 * T * TP) / 4;
    for (int k = threadIdx.x; k < n4; k += kDdeThreads) z4[k] = make_int4(0, 0, 0, 0);
  }
  const int64_t vbase = vis_off[l];
  const int32_t* toff = tile_off + (size_t)l * (ntr * ntc * 4 + 1);
  const int t0r = tr * T, t0c = tc * T;
  float S = 1.f;
  if (MODE == 0) {
    // sweep 0: bound m of the tap values of the visibilities meeting the tile; the
    // tile's own visibilities also get their scaled value written once
    float m = 0.f;
    for (int s = 0; s < 9; ++s) {
      const int src = dde_source(s, tr, tc, ntr, ntc);
      if (src < 0) continue;
      const bool own = src == tau;
      const int beg = toff[src * 4], end = toff[src * 4 + 4];
      for (int k = beg + (int)threadIdx.x; k < end; k += kDdeThreads) {
        const int64_t i = vbase + k;
        float2 val = vals[i];
        if (blk_scale) {
          const float sc = blk_scale[l * B + blk[i]];
          val.x *= sc;
          val.y *= sc;
        }
        if (own && v_write) v_write[i] = val;
        const float2 w = uv[i];
        float xr, xc;
        const int kr = kb_first(w.y, vg.tc.hi_r, vg.tc.lo_r, xr);
        const int kc = kb_first(w.x, vg.tc.hi_c, vg.tc.lo_c, xc);
        if (dde_meets(dde_local(kr - R, t0r, vg.K1, vg.pw), F, T, vg.K1) &&
            dde_meets(dde_local(kc - R, t0c, vg.K2, vg.pw), F, T, vg.K2))
          m = fmaxf(m, fmaxf(fabsf(val.x), fabsf(val.y)) * kl1[kidx[i]]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) sred[wid] = m;
    __syncthreads();
    m = 0.f;
#pragma unroll
    for (int w = 0; w < kDdeWarps; ++w) m = fmaxf(m, sred[w]);
    const int nc = ncmax[l * ntr * ntc + tau];
    if (m > 1e-30f && nc > 0) {
      const float t = 1073741824.f / ((float)nc * (m * 1.0009765625f));
      const int e = (int)((__float_as_uint(t) >> 23) & 0xffu) - 127;   // 2^e <= t
      S = pow2f(max(-120, min(e, 120)));
    }
  } else {
    __syncthreads();
  }
  // sweep 1: each warp takes 32 candidates at a time and processes the ones that meet
  // the tile, one by one
  for (int s = 0; s < 9; ++s) {
    const int src = dde_source(s, tr, tc, ntr, ntc);
    if (src < 0) continue;
    const int beg = toff[src * 4], end = toff[src * 4 + 4];
    for (int k0 = beg + wid * 32; k0 < end; k0 += kDdeThreads) {
      const int k = k0 + lane;
      bool hit = false;
      int dr = 0, dc = 0;
      float xr = 0.f, xc = 0.f;
      if (k < end) {
        const float2 w = uv[vbase + k];
        const int kr = kb_first(w.y, vg.tc.hi_r, vg.tc.lo_r, xr);
        const int kc = kb_first(w.x, vg.tc.hi_c, vg.tc.lo_c, xc);
        dr = dde_local(kr - R, t0r, vg.K1, vg.pw);
        dc = dde_local(kc - R, t0c, vg.K2, vg.pw);
        hit = dde_meets(dr, F, T, vg.K1) && dde_meets(dc, F, T, vg.K2);
      }
      unsigned mask = __ballot_sync(0xffffffffu, hit);
      while (mask) {
        const int src_lane = __ffs(mask) - 1;
        mask &= mask - 1;
        const int64_t i = vbase + k0 + src_lane;
        const int drs = __shfl_sync(0xffffffffu, dr, src_lane), dcs = __shfl_sync(0xffffffffu, dc, src_lane);
        const float xrs = __shfl_sync(0xffffffffu, xr, src_lane), xcs = __shfl_sync(0xffffffffu, xc, src_lane);
        float2 vS = make_float2(0.f, 0.f);
        const float2* Km = nullptr;
        if (MODE == 0) {
          float2 val = vals[i];
          const float sc = (blk_scale ? blk_scale[l * B + blk[i]] : 1.f) * S;
          vS = make_float2(val.x * sc, val.y * sc);
          Km = kern + (size_t)kidx[i] * SD * SD;
        }
        dde_grid_one<R, MODE>(are, aim, TP, T, drs, dcs, xrs, xcs, vS, Km, vg, scr[wid], lane);
      }
    }
  }
  __syncthreads();
  if (MODE == 1) {
    int mx = 0;
    for (int q = threadIdx.x; q < T * T; q += kDdeThreads) mx = max(mx, are[(q / T) * TP + q % T]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) sredi[wid] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 0; w < kDdeWarps; ++w) mx = max(mx, sredi[w]);
      ncmax[l * ntr * ntc + tau] = mx;
    }
    return;
  }
  const float inv = 1.f / S;                                   // power of two: exact
  float2* gl = grid + (size_t)l * vg.K1 * vg.K2;
  for (int q = threadIdx.x; q < T * T; q += kDdeThreads) {
    const int rr = q / T, cc = q % T, o = rr * TP + cc;
    const int row = phys_row2(t0r + rr, vg);
    gl[(size_t)row * vg.K2 + t0c + cc] = make_float2((float)are[o] * inv, (float)aim[o] * inv);
  }
}

// ------------------------------------------------------------- launchers
#define FHS_DDE_SWITCH(R, ...)                    \
  switch (R) {                                    \
    case 0: __VA_ARGS__(0); break;                \
    case 1: __VA_ARGS__(1); break;                \
    case 2: __VA_ARGS__(2); break;                \
    case 3: __VA_ARGS__(3); break;                \
    default: __VA_ARGS__(4); break;               \
  }

static size_t grid_dde_smem(const Cube& cb, int mode) {
  return (size_t)(mode == 1 ? 1 : 2) * cb.tile * grid_row_stride(cb.tile) * sizeof(int);
}

void launch_degrid_dde(const Cube& cb, const float2* grid, float2* out, cudaStream_t st) {
  dim3 grd(degrid_parts(cb), cb.L);
  const VisGeom vg = vis_geom(cb);
#define FHS_L(RR)                                                                                               \
  k_degrid_dde<RR, 0><<<grd, kDdeThreads, 0, st>>>(grid, cb.d_uv, cb.d_dde_kern, cb.d_dde_idx, cb.d_vis_off, vg, \
                                                   out, nullptr, nullptr, nullptr, nullptr, cb.B, nullptr, 0)
  FHS_DDE_SWITCH(cb.dde_R, FHS_L)
#undef FHS_L
  note_launches(1);
}

void launch_degrid_pdfb_dde(const Cube& cb, const float2* grid, const float2* y, const float2* v, float2* d_out,
                            float2* u_prev, double* partials, int nparts, cudaStream_t st) {
  dim3 grd(nparts, cb.L);
  const VisGeom vg = vis_geom(cb);
#define FHS_L(RR)                                                                                               \
  k_degrid_dde<RR, 1><<<grd, kDdeThreads, 0, st>>>(grid, cb.d_uv, cb.d_dde_kern, cb.d_dde_idx, cb.d_vis_off, vg, \
                                                   d_out, y, v, u_prev, cb.d_blk, cb.B, partials, nparts)
  FHS_DDE_SWITCH(cb.dde_R, FHS_L)
#undef FHS_L
  note_launches(1);
}

void launch_grid_dde(const Cube& cb, const float2* vals, const float* blk_scale, float2* v_write, float2* grid,
                     cudaStream_t st) {
  dim3 grd(cb.ntile_r * cb.ntile_c, cb.L);
  const VisGeom vg = vis_geom(cb);
  const size_t sm = grid_dde_smem(cb, 0);
  static bool attr[5] = {false, false, false, false, false};
#define FHS_L(RR)                                                                                                 \
  if (!attr[RR]) {                                                                                                \
    cudaFuncSetAttribute(k_grid_dde<RR, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 80 * 1024);               \
    attr[RR] = true;                                                                                              \
  }                                                                                                               \
  k_grid_dde<RR, 0><<<grd, kDdeThreads, sm, st>>>(vals, blk_scale, v_write, cb.d_uv, cb.d_blk, cb.d_dde_kern,      \
                                                  cb.d_dde_idx, cb.d_dde_l1, cb.d_tile_off, cb.d_vis_off, grid,   \
                                                  cb.d_dde_ncmax, vg, cb.tile, cb.ntile_r, cb.ntile_c, cb.B)
  FHS_DDE_SWITCH(cb.dde_R, FHS_L)
#undef FHS_L
  note_launches(1);
}

void launch_grid_dde_count(const Cube& cb, cudaStream_t st) {
  dim3 grd(cb.ntile_r * cb.ntile_c, cb.L);
  const VisGeom vg = vis_geom(cb);
  const size_t sm = grid_dde_smem(cb, 1);
  static bool attr[5] = {false, false, false, false, false};
#define FHS_L(RR)                                                                                                 \
  if (!attr[RR]) {                                                                                                \
    cudaFuncSetAttribute(k_grid_dde<RR, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 80 * 1024);               \
    attr[RR] = true;                                                                                              \
  }                                                                                                               \
  k_grid_dde<RR, 1><<<grd, kDdeThreads, sm, st>>>(nullptr, nullptr, nullptr, cb.d_uv, cb.d_blk, nullptr,           \
                                                  nullptr, nullptr, cb.d_tile_off, cb.d_vis_off, nullptr,         \
                                                  cb.d_dde_ncmax, vg, cb.tile, cb.ntile_r, cb.ntile_c, cb.B)
  FHS_DDE_SWITCH(cb.dde_R, FHS_L)
#undef FHS_L
  note_launches(1);
}

#undef FHS_DDE_SWITCH

}  // namespace fhs
