// k_sort.cu -- stable LSD radix sort of uint64 keys, exclusive scan, and the
// construction of the sorted (tile, Gaussian) pair list.
//
// The pair list is the tile list of the rasterizer: every visible (view,
// Gaussian) record is listed once per tile of its 3-sigma rectangle, tiles
// in global order, inside a tile by FP32 depth, ties by record index.
// Instead of one 64-bit sort of all pairs, the records are sorted by depth
// once (N keys, 4 passes) and the pairs emitted in that order are then
// sorted stably on the tile bits only (2-3 passes): the same order, with
// far fewer bytes moved per pair.
//
// Sort passes use reduce-then-scan (per-block digit histograms, a scan of
// them, a stable scatter).  No CTA ever waits for another one.
#include "cg_common.cuh"

namespace cg {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 keys per sort block
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr int kGrid = 152 * 8;

// ---------------------------------------------------------------------------
// radix sort
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kSortThreads) k_sort_upsweep(const uint64_t* __restrict__ keys,
                                                               const uint64_t* count_dev, int64_t count_cap,
                                                               int shift, uint32_t* __restrict__ hist,
                                                               int64_t nb_cap) {
  __shared__ uint32_t h[256];
  const int64_t count = min((int64_t)*count_dev, count_cap);
  const int64_t nb = (count + kSortTile - 1) / kSortTile;
  for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = b * kSortTile;
#pragma unroll 4
    for (int i = threadIdx.x; i < kSortTile; i += kSortThreads) {
      const int64_t idx = base + i;
      if (idx < count) atomicAdd(&h[(uint32_t)(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nb_cap + b] = h[threadIdx.x];
    __syncthreads();
  }
}

// Block-wide exclusive scan of one uint32 per thread (1024 threads max).
template <int NT>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_sums, uint32_t* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t s = lane < NT / 32 ? warp_sums[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < NT / 32) warp_sums[lane] = s;
  }
  __syncthreads();
  const uint32_t prefix = (wid > 0 ? warp_sums[wid - 1] : 0u) + x - v;
  if (total) *total = warp_sums[NT / 32 - 1];
  __syncthreads();
  return prefix;
}

// One CTA per digit: exclusive scan of that digit's per-block counts.
__global__ void __launch_bounds__(1024) k_sort_scan_rows(uint32_t* __restrict__ hist, const uint64_t* count_dev,
                                                         int64_t count_cap, int64_t nb_cap,
                                                         uint32_t* __restrict__ digit_tot) {
  __shared__ uint32_t ws[32];
  const int64_t count = min((int64_t)*count_dev, count_cap);
  const int64_t nb = (count + kSortTile - 1) / kSortTile;
  uint32_t* row = hist + (int64_t)blockIdx.x * nb_cap;
  uint32_t carry = 0;
  for (int64_t c = 0; c < nb; c += 1024) {
    const int64_t i = c + threadIdx.x;
    const uint32_t v = i < nb ? row[i] : 0u;
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan<1024>(v, ws, &tot);
    if (i < nb) row[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) digit_tot[blockIdx.x] = carry;
}

__global__ void __launch_bounds__(kSortThreads, 3) k_sort_downsweep(const uint64_t* __restrict__ in,
                                                                 uint64_t* __restrict__ out,
                                                                 const uint64_t* count_dev, int64_t count_cap,
                                                                 int shift, const uint32_t* __restrict__ hist,
                                                                 const uint32_t* __restrict__ digit_tot,
                                                                 int64_t nb_cap) {
  constexpr int kWarps = kSortThreads / 32;
  __shared__ uint64_t stage[kSortTile];
  __shared__ uint32_t wcnt[kWarps][256];
  __shared__ uint32_t digit_base[256];
  __shared__ uint32_t bstart[256];
  __shared__ uint32_t gbase[256];
  __shared__ uint32_t scan_ws[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t count = min((int64_t)*count_dev, count_cap);
  const int64_t nb = (count + kSortTile - 1) / kSortTile;
  // global start of each digit
  {
    const uint32_t t = digit_tot[threadIdx.x];
    digit_base[threadIdx.x] = block_exclusive_scan<kSortThreads>(t, scan_ws, nullptr);
  }
  const uint32_t lt_mask = (1u << lane) - 1u;
  for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
    for (int i = threadIdx.x; i < kWarps * 256; i += kSortThreads) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t base = b * kSortTile + (int64_t)wid * (32 * kSortItems);
    uint64_t key[kSortItems];
    uint32_t rank[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
      const int64_t idx = base + r * 32 + lane;
      const bool valid = idx < count;
      key[r] = valid ? in[idx] : 0ull;
      const uint32_t d = valid ? ((uint32_t)(key[r] >> shift) & 255u) : 256u;
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      const uint32_t before = __popc(peers & lt_mask);
      uint32_t old = 0;
      if (valid) old = wcnt[wid][d];
      __syncwarp();
      if (valid && before == 0) wcnt[wid][d] = old + __popc(peers);
      __syncwarp();
      rank[r] = old + before;
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, block count, block-local start
    {
      const int d = threadIdx.x;
      uint32_t acc = 0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = wcnt[w][d];
        wcnt[w][d] = acc;
        acc += c;
      }
      const uint32_t start = block_exclusive_scan<kSortThreads>(acc, scan_ws, nullptr);
      bstart[d] = start;
      gbase[d] = digit_base[d] + hist[(int64_t)d * nb_cap + b];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
      const int64_t idx = base + r * 32 + lane;
      if (idx < count) {
        const uint32_t d = (uint32_t)(key[r] >> shift) & 255u;
        stage[bstart[d] + wcnt[wid][d] + rank[r]] = key[r];
      }
    }
    __syncthreads();
    const int valid_n = (int)min((int64_t)kSortTile, count - b * kSortTile);
    for (int i = threadIdx.x; i < valid_n; i += kSortThreads) {
      const uint64_t k = stage[i];
      const uint32_t d = (uint32_t)(k >> shift) & 255u;
      out[gbase[d] + (uint32_t)i - bstart[d]] = k;
    }
    __syncthreads();
  }
}

cudaError_t sort_u64(void* ws, const Layout& L, uint64_t* a, uint64_t* b, const uint64_t* count_dev,
                     int64_t count_cap, int lo_bit, int passes, bool* result_in_b, cudaStream_t s) {
  uint32_t* hist = ws_ptr<uint32_t>(ws, L.hist);
  uint32_t* digit_tot = hist + 256 * L.sort_blocks_cap;
  const int64_t nb_cap = (count_cap + kSortTile - 1) / kSortTile;
  if (nb_cap > L.sort_blocks_cap) return cudaErrorInvalidValue;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(nb_cap, kGrid));
  uint64_t* src = a;
  uint64_t* dst = b;
  for (int p = 0; p < passes; ++p) {
    const int shift = lo_bit + 8 * p;
    count_launch(), k_sort_upsweep<<<grid, kSortThreads, 0, s>>>(src, count_dev, count_cap, shift, hist, L.sort_blocks_cap);
    count_launch(), k_sort_scan_rows<<<256, 1024, 0, s>>>(hist, count_dev, count_cap, L.sort_blocks_cap, digit_tot);
    count_launch(), k_sort_downsweep<<<grid, kSortThreads, 0, s>>>(src, dst, count_dev, count_cap, shift, hist, digit_tot,
                                                   L.sort_blocks_cap);
    uint64_t* t = src;
    src = dst;
    dst = t;
  }
  *result_in_b = (passes & 1) != 0;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// exclusive scan of uint32 values (64-bit block sums and total)
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ in,
                                                              const uint64_t* count_dev, int64_t count_cap,
                                                              uint64_t* __restrict__ bsum) {
  __shared__ uint64_t red[kScanThreads / 32];
  const int64_t count = min((int64_t)*count_dev, count_cap);
  const int64_t nb = (count + kScanTile - 1) / kScanTile;
  for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
    uint64_t acc = 0;
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
      const int64_t idx = b * kScanTile + i;
      if (idx < count) acc += in[idx];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint64_t t = 0;
      for (int w = 0; w < kScanThreads / 32; ++w) t += red[w];
      bsum[b] = t;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(1024) k_scan_blocks(uint64_t* __restrict__ bsum, const uint64_t* count_dev,
                                                      int64_t count_cap, uint64_t* total_dev) {
  __shared__ uint64_t wsum[32];
  const int64_t count = min((int64_t)*count_dev, count_cap);
  const int64_t nb = (count + kScanTile - 1) / kScanTile;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint64_t carry = 0;
  for (int64_t c = 0; c < nb; c += 1024) {
    const int64_t i = c + threadIdx.x;
    const uint64_t v = i < nb ? bsum[i] : 0ull;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
      uint64_t sw = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, sw, o);
        if (lane >= o) sw += y;
      }
      wsum[lane] = sw;
    }
    __syncthreads();
    const uint64_t ex = (wid > 0 ? wsum[wid - 1] : 0ull) + x - v;
    if (i < nb) bsum[i] = carry + ex;
    const uint64_t tot = wsum[31];
    __syncthreads();
    carry += tot;
  }
  if (threadIdx.x == 0) *total_dev = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const uint32_t* in, uint32_t* out,
                                                            const uint64_t* count_dev, int64_t count_cap,
                                                            const uint64_t* __restrict__ bsum) {
  __shared__ uint32_t ws[32];
  const int64_t count = min((int64_t)*count_dev, count_cap);
  const int64_t nb = (count + kScanTile - 1) / kScanTile;
  for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
    // blocked arrangement: thread t owns items [t*16, t*16+16)
    const int64_t base = b * kScanTile + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t local = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
      v[i] = base + i < count ? in[base + i] : 0u;
      local += v[i];
    }
    const uint32_t pre = block_exclusive_scan<kScanThreads>(local, ws, nullptr);
    uint32_t run = (uint32_t)bsum[b] + pre;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
      if (base + i < count) out[base + i] = run;
      run += v[i];
    }
    __syncthreads();
  }
}

cudaError_t scan_u32(void* ws, const Layout& L, const uint32_t* in, uint32_t* out, const uint64_t* count_dev,
                     int64_t count_cap, uint64_t* total_dev, cudaStream_t s) {
  uint64_t* bsum = ws_ptr<uint64_t>(ws, L.blocksums);
  const int64_t nb_cap = (count_cap + kScanTile - 1) / kScanTile;
  if (nb_cap > L.scan_blocks_cap) return cudaErrorInvalidValue;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(nb_cap, kGrid));
  count_launch(), k_scan_reduce<<<grid, kScanThreads, 0, s>>>(in, count_dev, count_cap, bsum);
  count_launch(), k_scan_blocks<<<1, 1024, 0, s>>>(bsum, count_dev, count_cap, total_dev);
  count_launch(), k_scan_down<<<grid, kScanThreads, 0, s>>>(in, out, count_dev, count_cap, bsum);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// pair list
// ---------------------------------------------------------------------------

__global__ void k_visible_flags(const uint32_t* __restrict__ ntiles, uint32_t* __restrict__ flags, int64_t R,
                                uint64_t* count_slot) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < R; i += stride)
    flags[i] = ntiles[i] > 0 ? 1u : 0u;
  if (blockIdx.x == 0 && threadIdx.x == 0) *count_slot = (uint64_t)R;
}

__global__ void k_compact_depth(const uint32_t* __restrict__ ntiles, const uint32_t* __restrict__ depth,
                                const uint32_t* __restrict__ pos, uint64_t* __restrict__ dkeys, int64_t R) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < R; i += stride)
    if (ntiles[i] > 0) dkeys[pos[i]] = ((uint64_t)depth[i] << 32) | (uint64_t)i;
}

__global__ void k_gather_ntiles(const uint64_t* __restrict__ dkeys, const uint32_t* __restrict__ ntiles,
                                uint32_t* __restrict__ out, const uint64_t* visible_dev) {
  const int64_t vis = (int64_t)*visible_dev;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < vis; i += stride)
    out[i] = ntiles[(uint32_t)dkeys[i]];
}

__global__ void k_capacity(DeviceState* st, int64_t cap) {
  const uint64_t k = st->scan_total;
  st->pairs = k;
  const bool ok = k <= (uint64_t)cap;
  st->pairs_ok = ok ? 1u : 0u;
  st->pad = 0;
  if (!ok) set_status(st, CG_ERR_CAPACITY, 0);
}

// Pairs of one record: (global tile << 32) | record, tiles of its rectangle
// in row-major order starting at its offset.  A warp takes 32 consecutive
// records (depth order) and writes their pairs one record at a time with all
// lanes, so the stores of a record are contiguous.
__global__ void __launch_bounds__(256) k_emit_pairs(const uint64_t* __restrict__ dkeys,
                                                    const uint32_t* __restrict__ off_sorted,
                                                    const ushort4* __restrict__ rect,
                                                    const ViewInfo* __restrict__ views, int64_t n,
                                                    uint32_t* __restrict__ offrec, uint64_t* __restrict__ pairs,
                                                    const DeviceState* st) {
  const int64_t vis = (int64_t)st->visible;
  const bool ok = st->pairs_ok != 0;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base = warp * 32; base < vis; base += nwarps * 32) {
    const int64_t i = base + lane;
    uint32_t rec = 0, off = 0, r01 = 0, r23 = 0;
    if (i < vis) {
      rec = (uint32_t)dkeys[i];
      off = off_sorted[i];
      offrec[rec] = off;
      const ushort4 r = rect[rec];
      r01 = (uint32_t)r.x | ((uint32_t)r.y << 16);
      r23 = (uint32_t)r.z | ((uint32_t)r.w << 16);
    }
    if (!ok) continue;
    const int cnt = (int)min((int64_t)32, vis - base);
    for (int q = 0; q < cnt; ++q) {
      const uint32_t qrec = __shfl_sync(0xffffffffu, rec, q);
      const uint32_t qoff = __shfl_sync(0xffffffffu, off, q);
      const uint32_t q01 = __shfl_sync(0xffffffffu, r01, q);
      const uint32_t q23 = __shfl_sync(0xffffffffu, r23, q);
      const int x0 = (int)(q01 & 0xffffu), y0 = (int)(q01 >> 16);
      const int w = (int)(q23 & 0xffffu) - x0, h = (int)(q23 >> 16) - y0;
      const ViewInfo& cam = views[qrec / (uint64_t)n];
      const int64_t tb = cam.tile_base;
      const int tx = cam.tiles_x;
      const int total = w * h;
      for (int t = lane; t < total; t += 32) {
        const int yy = t / w, xx = t - yy * w;
        pairs[qoff + t] = ((uint64_t)(tb + (int64_t)(y0 + yy) * tx + (x0 + xx)) << 32) | qrec;
      }
    }
  }
}

__global__ void k_zero_u32(uint32_t* p, int64_t count) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) p[i] = 0u;
}

__global__ void k_ranges(const uint64_t* __restrict__ pairs, uint2* __restrict__ ranges, const DeviceState* st) {
  const int64_t k = st->pairs_ok ? (int64_t)st->pairs : 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += stride) {
    const uint32_t t = (uint32_t)(pairs[i] >> 32);
    if (i == 0 || (uint32_t)(pairs[i - 1] >> 32) != t) ranges[t].x = (uint32_t)i;
    if (i == k - 1 || (uint32_t)(pairs[i + 1] >> 32) != t) ranges[t].y = (uint32_t)(i + 1);
  }
}

cudaError_t launch_build_pairs(const Layout& L, void* ws, int tile_bits, cudaStream_t s) {
  WsHeader* hdr = ws_ptr<WsHeader>(ws, L.hdr);
  DeviceState* st = &hdr->st;
  const uint32_t* ntiles = ws_ptr<uint32_t>(ws, L.ntiles);
  const uint32_t* depth = ws_ptr<uint32_t>(ws, L.depth);
  uint32_t* scan = ws_ptr<uint32_t>(ws, L.scan);
  uint64_t* dk0 = ws_ptr<uint64_t>(ws, L.dkeys0);
  uint64_t* dk1 = ws_ptr<uint64_t>(ws, L.dkeys1);
  const int64_t R = L.R;
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>((R + 255) / 256, kGrid));
  // 1. compact visible records, keyed by FP32 depth bits (record index low)
  count_launch(), k_visible_flags<<<g, 256, 0, s>>>(ntiles, scan, R, &st->scan_total);
  cudaError_t e = scan_u32(ws, L, scan, scan, &st->scan_total, R, &st->visible, s);
  if (e != cudaSuccess) return e;
  count_launch(), k_compact_depth<<<g, 256, 0, s>>>(ntiles, depth, scan, dk0, R);
  // 2. stable sort by depth (records in index order for equal depth)
  bool in_b = false;
  e = sort_u64(ws, L, dk0, dk1, &st->visible, R, 32, 4, &in_b, s);
  if (e != cudaSuccess) return e;
  const uint64_t* dsorted = in_b ? dk1 : dk0;
  if (dsorted != depth_sorted(ws, L)) return cudaErrorInvalidValue;
  // 3. pair offsets in depth order, total pair count and capacity check
  count_launch(), k_gather_ntiles<<<g, 256, 0, s>>>(dsorted, ntiles, scan, &st->visible);
  e = scan_u32(ws, L, scan, scan, &st->visible, R, &st->scan_total, s);
  if (e != cudaSuccess) return e;
  count_launch(), k_capacity<<<1, 1, 0, s>>>(st, L.Kc);
  // 4. emit pairs in depth order
  uint64_t* p0 = ws_ptr<uint64_t>(ws, L.pairs0);
  uint64_t* p1 = ws_ptr<uint64_t>(ws, L.pairs1);
  count_launch(), k_emit_pairs<<<g, 256, 0, s>>>(dsorted, scan, ws_ptr<const ushort4>(ws, L.rect), ws_ptr<ViewInfo>(ws, L.views),
                                 L.n, ws_ptr<uint32_t>(ws, L.offrec), p0, st);
  // 5. stable sort on the tile bits
  const int passes = (tile_bits + 7) / 8;
  e = sort_u64(ws, L, p0, p1, &st->pairs, L.Kc, 32, passes, &in_b, s);
  if (e != cudaSuccess) return e;
  const uint64_t* psorted = in_b ? p1 : p0;
  // 6. per-tile ranges
  uint2* ranges = ws_ptr<uint2>(ws, L.ranges);
  const int gt = (int)std::max<int64_t>(1, std::min<int64_t>((2 * L.T + 255) / 256, kGrid));
  count_launch(), k_zero_u32<<<gt, 256, 0, s>>>(reinterpret_cast<uint32_t*>(ranges), 2 * L.T);
  const int gk = (int)std::max<int64_t>(1, std::min<int64_t>((L.Kc + 255) / 256, kGrid));
  count_launch(), k_ranges<<<gk, 256, 0, s>>>(psorted, ranges, st);
  return cudaGetLastError();
}

}  // namespace cg
