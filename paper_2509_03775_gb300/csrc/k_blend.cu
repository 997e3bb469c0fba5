// k_blend.cu -- per-tile compositing of Eq. 3 (forward) and its reverse
// (backward), one CTA per tile.
//
// Forward: the tile's sorted Gaussians are staged in shared memory in
// batches; every thread walks them front to back for its pixel(s) with the
// decision arithmetic (skip alpha < 1/255, clamp at 0.99, stop before the
// transmittance would fall below 1e-4), and writes the colour, the final
// transmittance and the position after the last contributor.
//
// Backward: the tile's list is walked back to front from the largest
// contributor position of the tile.  Each pixel recomputes alpha with the
// same arithmetic (so it takes the forward's decisions exactly) and
// undoes the transmittance by division.  The nine per-pixel gradient terms of
// every (tile, Gaussian) pair -- mean x/y, conic 0/1/2, opacity, colour
// r/g/b -- are summed over the tile's pixels in a fixed order (registers,
// warp butterfly, warps in index order) and written to the pair's slot, so
// the per-Gaussian gradient later sums a fixed set of slots in a fixed order.
#include <algorithm>

#include "cg_common.cuh"

namespace cg {

struct BlendGeo {
  float4 a;  // mean x, mean y, h0, h1
  float4 b;  // h2, opacity, skip bound, 0
};

// power = h0 dx^2 + h1 dx dy + h2 dy^2 with d = mean - pixel centre
// (decision arithmetic).
__device__ __forceinline__ float gauss_power(const float4& a, const float4& b, float pxc, float pyc, float& dx,
                                             float& dy) {
  dx = a.x - pxc;
  dy = a.y - pyc;
  return fmaf(a.z * dx, dx, fmaf(b.x * dy, dy, (a.w * dx) * dy));
}

template <int TILE, int BATCH>
__global__ void __launch_bounds__(TILE* TILE < 256 ? TILE* TILE : 256)
    k_blend_fwd(const ViewInfo* __restrict__ views, int n_views, const uint2* __restrict__ ranges,
                const uint64_t* __restrict__ pairs, const float4* __restrict__ geo, const float4* __restrict__ rgbm,
                float bg0, float bg1, float bg2, float* __restrict__ images, float* __restrict__ tfinal,
                uint32_t* __restrict__ ncontrib) {
  constexpr int NT = TILE * TILE < 256 ? TILE * TILE : 256;
  constexpr int PPT = TILE * TILE / NT;
  __shared__ float4 sA[BATCH], sB[BATCH], sC[BATCH];
  const int64_t gt = blockIdx.x;
  const int v = find_view(views, n_views, gt);
  const ViewInfo& cam = views[v];
  const int64_t lt = gt - cam.tile_base;
  const int tx = (int)(lt % cam.tiles_x), ty = (int)(lt / cam.tiles_x);
  const uint2 rg = ranges[gt];
  float pxc[PPT], pyc[PPT], T[PPT], C[PPT][3];
  uint32_t last[PPT];
  bool done[PPT];
  int px[PPT], py[PPT];
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int p = threadIdx.x + k * NT;
    px[k] = tx * TILE + p % TILE;
    py[k] = ty * TILE + p / TILE;
    pxc[k] = (float)px[k] + 0.5f;
    pyc[k] = (float)py[k] + 0.5f;
    T[k] = 1.0f;
    C[k][0] = C[k][1] = C[k][2] = 0.0f;
    last[k] = 0;
    done[k] = !(px[k] < cam.width && py[k] < cam.height);
  }
  for (uint32_t b0 = rg.x; b0 < rg.y; b0 += BATCH) {
    bool mine = true;
#pragma unroll
    for (int k = 0; k < PPT; ++k) mine = mine && done[k];
    if (__syncthreads_and(mine)) break;
    const int n_in = (int)min((uint32_t)BATCH, rg.y - b0);
    for (int j = threadIdx.x; j < n_in; j += NT) {
      const uint32_t rec = (uint32_t)pairs[b0 + j];
      sA[j] = geo[2 * (size_t)rec];
      sB[j] = geo[2 * (size_t)rec + 1];
      sC[j] = rgbm[rec];
    }
    __syncthreads();
    for (int j = 0; j < n_in; ++j) {
      const float4 a = sA[j], b = sB[j];
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        if (done[k]) continue;
        float dx, dy;
        const float power = gauss_power(a, b, pxc[k], pyc[k], dx, dy);
        if (power > 0.0f || power < b.z) continue;
        const float vv = b.y * exp32(power);
        const float alpha = vv > kAlphaMax ? kAlphaMax : vv;
        if (alpha < kAlphaMin) continue;
        const float test_T = T[k] * (1.0f - alpha);
        if (test_T < kTMin) {
          done[k] = true;
          continue;
        }
        const float4 c = sC[j];
        const float w = alpha * T[k];
        C[k][0] = fmaf(w, c.x, C[k][0]);
        C[k][1] = fmaf(w, c.y, C[k][1]);
        C[k][2] = fmaf(w, c.z, C[k][2]);
        T[k] = test_T;
        last[k] = b0 - rg.x + j + 1;
      }
    }
  }
  const int64_t hw = (int64_t)cam.width * cam.height;
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    if (!(px[k] < cam.width && py[k] < cam.height)) continue;
    const int64_t pix = cam.pix_base + (int64_t)py[k] * cam.width + px[k];
    float* img = images + 3 * cam.pix_base + (int64_t)py[k] * cam.width + px[k];
    img[0] = fmaf(T[k], bg0, C[k][0]);
    img[hw] = fmaf(T[k], bg1, C[k][1]);
    img[2 * hw] = fmaf(T[k], bg2, C[k][2]);
    tfinal[pix] = T[k];
    ncontrib[pix] = last[k];
  }
}

template <int TILE, int BATCH>
__global__ void __launch_bounds__(TILE* TILE < 256 ? TILE* TILE : 256)
    k_blend_bwd(const ViewInfo* __restrict__ views, int n_views, const uint2* __restrict__ ranges,
                const uint64_t* __restrict__ pairs, const float4* __restrict__ geo, const float4* __restrict__ rgbm,
                const ushort4* __restrict__ rect, const uint32_t* __restrict__ offrec, float bg0, float bg1,
                float bg2, const float* __restrict__ d_images, const float* __restrict__ tfinal,
                const uint32_t* __restrict__ ncontrib, float* __restrict__ pairgrad) {
  constexpr int NT = TILE * TILE < 256 ? TILE * TILE : 256;
  constexpr int PPT = TILE * TILE / NT;
  constexpr int NW = NT / 32;
  __shared__ float4 sA[BATCH], sB[BATCH], sC[BATCH];
  __shared__ uint32_t sSlot[BATCH];
  __shared__ float part[NW][BATCH][9];
  __shared__ uint32_t s_maxc;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t gt = blockIdx.x;
  const int v = find_view(views, n_views, gt);
  const ViewInfo& cam = views[v];
  const int64_t lt = gt - cam.tile_base;
  const int tx = (int)(lt % cam.tiles_x), ty = (int)(lt / cam.tiles_x);
  const uint2 rg = ranges[gt];
  const int64_t hw = (int64_t)cam.width * cam.height;
  float pxc[PPT], pyc[PPT], T[PPT], tfin[PPT], dC[PPT][3], acc[PPT][3], bgdot[PPT];
  uint32_t nc[PPT];
  if (threadIdx.x == 0) s_maxc = 0;
  __syncthreads();
  uint32_t my_max = 0;
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int p = threadIdx.x + k * NT;
    const int x = tx * TILE + p % TILE, y = ty * TILE + p / TILE;
    pxc[k] = (float)x + 0.5f;
    pyc[k] = (float)y + 0.5f;
    acc[k][0] = acc[k][1] = acc[k][2] = 0.0f;
    if (x < cam.width && y < cam.height) {
      const int64_t pix = cam.pix_base + (int64_t)y * cam.width + x;
      const float* dimg = d_images + 3 * cam.pix_base + (int64_t)y * cam.width + x;
      dC[k][0] = dimg[0];
      dC[k][1] = dimg[hw];
      dC[k][2] = dimg[2 * hw];
      tfin[k] = tfinal[pix];
      nc[k] = ncontrib[pix];
    } else {
      dC[k][0] = dC[k][1] = dC[k][2] = 0.0f;
      tfin[k] = 1.0f;
      nc[k] = 0;
    }
    T[k] = tfin[k];
    bgdot[k] = tfin[k] * fmaf(bg0, dC[k][0], fmaf(bg1, dC[k][1], bg2 * dC[k][2]));
    my_max = max(my_max, nc[k]);
  }
  atomicMax(&s_maxc, my_max);
  __syncthreads();
  const uint32_t maxc = s_maxc;
  const uint32_t len = rg.y - rg.x;
  // pairs past the last contributor of every pixel get zero gradient
  for (uint32_t j = maxc + threadIdx.x; j < len; j += NT) {
    const uint32_t rec = (uint32_t)pairs[rg.x + j];
    const ushort4 r = rect[rec];
    const uint32_t slot = offrec[rec] + (uint32_t)(ty - r.y) * (uint32_t)(r.z - r.x) + (uint32_t)(tx - r.x);
#pragma unroll
    for (int e = 0; e < 9; ++e) pairgrad[9 * (size_t)slot + e] = 0.0f;
  }
  // batches from the back: [b0, b1) with b1 - rg.x a multiple of BATCH except the first
  for (int64_t b1 = (int64_t)rg.x + maxc; b1 > (int64_t)rg.x; b1 -= BATCH) {
    const int64_t b0 = max((int64_t)rg.x, b1 - BATCH);
    const int n_in = (int)(b1 - b0);
    __syncthreads();
    for (int j = threadIdx.x; j < n_in; j += NT) {
      const uint32_t rec = (uint32_t)pairs[b0 + j];
      sA[j] = geo[2 * (size_t)rec];
      sB[j] = geo[2 * (size_t)rec + 1];
      sC[j] = rgbm[rec];
      const ushort4 r = rect[rec];
      sSlot[j] = offrec[rec] + (uint32_t)(ty - r.y) * (uint32_t)(r.z - r.x) + (uint32_t)(tx - r.x);
    }
    __syncthreads();
    for (int j = n_in - 1; j >= 0; --j) {
      const float4 a = sA[j], b = sB[j], c = sC[j];
      const uint32_t pos = (uint32_t)(b0 - rg.x) + j;
      float g[9];
#pragma unroll
      for (int e = 0; e < 9; ++e) g[e] = 0.0f;
      bool any = false;
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        if (pos >= nc[k]) continue;
        float dx, dy;
        const float power = gauss_power(a, b, pxc[k], pyc[k], dx, dy);
        if (power > 0.0f || power < b.z) continue;
        const float ex = exp32(power);
        const float vv = b.y * ex;
        const bool clamped = vv > kAlphaMax;
        const float alpha = clamped ? kAlphaMax : vv;
        if (alpha < kAlphaMin) continue;
        any = true;
        const float om = 1.0f - alpha;
        const float Tk = __fdividef(T[k], om);
        const float w = alpha * Tk;
        g[6] = fmaf(w, dC[k][0], g[6]);
        g[7] = fmaf(w, dC[k][1], g[7]);
        g[8] = fmaf(w, dC[k][2], g[8]);
        const float dot = fmaf(c.x - acc[k][0], dC[k][0], fmaf(c.y - acc[k][1], dC[k][1], (c.z - acc[k][2]) * dC[k][2]));
        const float dalpha = Tk * dot - __fdividef(bgdot[k], om);
        if (!clamped) {
          const float dpow = alpha * dalpha;
          g[0] = fmaf(dpow, fmaf(2.0f * a.z, dx, a.w * dy), g[0]);
          g[1] = fmaf(dpow, fmaf(2.0f * b.x, dy, a.w * dx), g[1]);
          g[2] = fmaf(dpow, -0.5f * dx * dx, g[2]);
          g[3] = fmaf(dpow, -dx * dy, g[3]);
          g[4] = fmaf(dpow, -0.5f * dy * dy, g[4]);
          g[5] = fmaf(ex, dalpha, g[5]);
        }
        acc[k][0] = fmaf(alpha, c.x - acc[k][0], acc[k][0]);
        acc[k][1] = fmaf(alpha, c.y - acc[k][1], acc[k][1]);
        acc[k][2] = fmaf(alpha, c.z - acc[k][2], acc[k][2]);
        T[k] = Tk;
      }
      if (__any_sync(0xffffffffu, any)) {
#pragma unroll
        for (int e = 0; e < 9; ++e) {
          float x = g[e];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
          g[e] = x;
        }
      }
      if (lane == 0) {
#pragma unroll
        for (int e = 0; e < 9; ++e) part[wid][j][e] = g[e];
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n_in * 9; i += NT) {
      const int j = i / 9, e = i - 9 * j;
      float s = 0.0f;
#pragma unroll
      for (int w = 0; w < NW; ++w) s += part[w][j][e];
      pairgrad[9 * (size_t)sSlot[j] + e] = s;
    }
  }
}

template <int TILE>
static cudaError_t fwd_tile(int batch, dim3 grid, cudaStream_t s, const ViewInfo* views, int nv, const uint2* rg,
                            const uint64_t* pairs, const float4* geo, const float4* rgbm, const float* bg,
                            float* images, float* tfinal, uint32_t* ncontrib) {
  constexpr int NT = TILE * TILE < 256 ? TILE * TILE : 256;
  switch (batch) {
    case 32: count_launch(), k_blend_fwd<TILE, 32><<<grid, NT, 0, s>>>(views, nv, rg, pairs, geo, rgbm, bg[0], bg[1], bg[2], images, tfinal, ncontrib); break;
    case 64: count_launch(), k_blend_fwd<TILE, 64><<<grid, NT, 0, s>>>(views, nv, rg, pairs, geo, rgbm, bg[0], bg[1], bg[2], images, tfinal, ncontrib); break;
    case 128: count_launch(), k_blend_fwd<TILE, 128><<<grid, NT, 0, s>>>(views, nv, rg, pairs, geo, rgbm, bg[0], bg[1], bg[2], images, tfinal, ncontrib); break;
    case 256: count_launch(), k_blend_fwd<TILE, 256><<<grid, NT, 0, s>>>(views, nv, rg, pairs, geo, rgbm, bg[0], bg[1], bg[2], images, tfinal, ncontrib); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int TILE>
static cudaError_t bwd_tile(int batch, dim3 grid, cudaStream_t s, const ViewInfo* views, int nv, const uint2* rg,
                            const uint64_t* pairs, const float4* geo, const float4* rgbm, const ushort4* rect,
                            const uint32_t* offrec, const float* bg, const float* d_images, const float* tfinal,
                            const uint32_t* ncontrib, float* pairgrad) {
  constexpr int NT = TILE * TILE < 256 ? TILE * TILE : 256;
  switch (batch) {
    case 32: count_launch(), k_blend_bwd<TILE, 32><<<grid, NT, 0, s>>>(views, nv, rg, pairs, geo, rgbm, rect, offrec, bg[0], bg[1], bg[2], d_images, tfinal, ncontrib, pairgrad); break;
    case 64: count_launch(), k_blend_bwd<TILE, 64><<<grid, NT, 0, s>>>(views, nv, rg, pairs, geo, rgbm, rect, offrec, bg[0], bg[1], bg[2], d_images, tfinal, ncontrib, pairgrad); break;
    case 128: count_launch(), k_blend_bwd<TILE, 128><<<grid, NT, 0, s>>>(views, nv, rg, pairs, geo, rgbm, rect, offrec, bg[0], bg[1], bg[2], d_images, tfinal, ncontrib, pairgrad); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

static const uint64_t* final_pairs(const Layout& L, void* ws) {
  const int passes = (L.tile_bits + 7) / 8;
  return (passes & 1) ? ws_ptr<const uint64_t>(ws, L.pairs1) : ws_ptr<const uint64_t>(ws, L.pairs0);
}

cudaError_t launch_blend_fwd(const Layout& L, void* ws, int tile, int batch, const float bg[3], float* images,
                             cudaStream_t s) {
  if (L.T <= 0) return cudaSuccess;
  const dim3 grid((unsigned)L.T);
  const ViewInfo* views = ws_ptr<ViewInfo>(ws, L.views);
  const uint2* rg = ws_ptr<uint2>(ws, L.ranges);
  const float4* geo = ws_ptr<float4>(ws, L.geo);
  const float4* rgbm = ws_ptr<float4>(ws, L.rgbm);
  float* tf = ws_ptr<float>(ws, L.tfinal);
  uint32_t* nc = ws_ptr<uint32_t>(ws, L.ncontrib);
  const uint64_t* pairs = final_pairs(L, ws);
  switch (tile) {
    case 8: return fwd_tile<8>(batch, grid, s, views, L.n_views, rg, pairs, geo, rgbm, bg, images, tf, nc);
    case 16: return fwd_tile<16>(batch, grid, s, views, L.n_views, rg, pairs, geo, rgbm, bg, images, tf, nc);
    case 32: return fwd_tile<32>(batch, grid, s, views, L.n_views, rg, pairs, geo, rgbm, bg, images, tf, nc);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_blend_bwd(const Layout& L, void* ws, int tile, int batch, const float bg[3],
                             const float* d_images, cudaStream_t s) {
  if (L.T <= 0) return cudaSuccess;
  const dim3 grid((unsigned)L.T);
  const ViewInfo* views = ws_ptr<ViewInfo>(ws, L.views);
  const uint2* rg = ws_ptr<uint2>(ws, L.ranges);
  const float4* geo = ws_ptr<float4>(ws, L.geo);
  const float4* rgbm = ws_ptr<float4>(ws, L.rgbm);
  const ushort4* rect = ws_ptr<ushort4>(ws, L.rect);
  const uint32_t* offrec = ws_ptr<uint32_t>(ws, L.offrec);
  const float* tf = ws_ptr<float>(ws, L.tfinal);
  const uint32_t* nc = ws_ptr<uint32_t>(ws, L.ncontrib);
  float* pg = ws_ptr<float>(ws, L.pairgrad);
  const uint64_t* pairs = final_pairs(L, ws);
  const int bb = batch > 128 ? 128 : batch;
  switch (tile) {
    case 8: return bwd_tile<8>(bb, grid, s, views, L.n_views, rg, pairs, geo, rgbm, rect, offrec, bg, d_images, tf, nc, pg);
    case 16: return bwd_tile<16>(bb, grid, s, views, L.n_views, rg, pairs, geo, rgbm, rect, offrec, bg, d_images, tf, nc, pg);
    case 32: return bwd_tile<32>(bb, grid, s, views, L.n_views, rg, pairs, geo, rgbm, rect, offrec, bg, d_images, tf, nc, pg);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace cg
