// Tile binning and sorting for the tile-based rasteriser (no CUB). The pair order is that of the
// 64-bit key (tile id << 32 | depth bits), ties in record order, built in three steps:
//   1. each visible record counts the tiles its footprint ellipse reaches; a scan over records
//      gives every record its range of pair slots;
//   2. duplication writes each (tile, record) pair into its slot and takes the pair's rank within
//      its tile from an atomic per-tile counter; a scan over the tile counts gives each tile its
//      range of the output (the tile ranges) and the pairs are scattered into their tile's range
//      as 64-bit keys (depth bits << 32 | record);
//   3. every tile's keys are sorted in shared memory (one CTA per tile, an ascending bitonic
//      network on the padded list; long lists go to a second kernel with a larger shared buffer, or
//      to the same network run in global memory), which orders the tile by (depth, record) no
//      matter in which order the atomics ranked its pairs.
//
// Every kernel reads its item count from device memory and sizes its work from it, so the
// whole sequence needs no host synchronisation and can be captured in a CUDA graph; grids are
// launched for the capacity and surplus blocks exit at once.
#include "common.cuh"

namespace dass {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;   // 2048 elements per scan block

constexpr int kSortThreads = 512;         // threads of the per-tile sort CTA
constexpr int kSortCap = 4096;            // longest tile list sorted by the per-tile kernel (32 KB)
constexpr int kBigThreads = 1024;
constexpr int kBigCap = 16384;            // longest list sorted in shared memory by the big-tile kernel (128 KB)
constexpr int kBigBlocks = 152;

// ----------------------------------------------------------------- exclusive scan (u32 -> u32)
// Three passes: per-block sums, one-block scan of the sums (64-bit, also writes the total),
// per-block scan with the block's offset. Length comes from *len (device).

__global__ void scan_reduce_kernel(const uint32_t* __restrict__ in, const long long* len_dev,
                                   unsigned long long* __restrict__ partial) {
    long long len = *len_dev;
    long long base = (long long)blockIdx.x * kScanTile;
    if (base >= len) return;
    unsigned long long s = 0;
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        long long idx = base + i;
        if (idx < len) s += in[idx];
    }
    __shared__ unsigned long long red[kScanThreads / 32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) t += red[w];
        partial[blockIdx.x] = t;
    }
}

// One block of 1024 threads scans nb partials in place (exclusive) and writes the total.
__global__ void scan_partials_kernel(unsigned long long* partial, const long long* len_dev,
                                     long long* total_out) {
    long long len = *len_dev;
    int nb = (int)((len + kScanTile - 1) / kScanTile);
    __shared__ unsigned long long sh[1024];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += 1024) {
        int i = base + threadIdx.x;
        unsigned long long v = i < nb ? partial[i] : 0ull;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            unsigned long long t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0ull;
            __syncthreads();
            sh[threadIdx.x] += t;
            __syncthreads();
        }
        unsigned long long incl = sh[threadIdx.x];
        if (i < nb) partial[i] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += incl;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total_out) *total_out = (long long)carry;
}

__global__ void scan_down_kernel(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                 const long long* len_dev, const unsigned long long* __restrict__ partial) {
    long long len = *len_dev;
    long long base = (long long)blockIdx.x * kScanTile;
    if (base >= len) return;
    // blocked arrangement: thread t owns items [t*8, t*8+8)
    uint32_t v[kScanItems];
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        long long idx = base + threadIdx.x * kScanItems + k;
        v[k] = idx < len ? in[idx] : 0u;
        sum += v[k];
    }
    __shared__ uint32_t wsum[kScanThreads / 32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint32_t woff = 0;
    for (int w = 0; w < warp; ++w) woff += wsum[w];
    uint32_t run = (uint32_t)partial[blockIdx.x] + woff + incl - sum;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        long long idx = base + threadIdx.x * kScanItems + k;
        if (idx < len) out[idx] = run;
        run += v[k];
    }
}

// ----------------------------------------------------------------- binning kernels

// Record -> (depth key, own index, number of tiles whose pixel centres the footprint ellipse
// reaches). A visible record has radius > 0; its candidate tile rows come from the ellipse's
// bounding box and each row contributes the contiguous run of tiles its band of the ellipse
// reaches (exact, conservative).
__device__ __forceinline__ bool record_footprint(const dass_splat* __restrict__ splats, long long rec, Footprint& f,
                                                 float& depth) {
    const float4* sp = reinterpret_cast<const float4*>(splats + rec);
    float4 s0 = __ldg(sp);
    float4 s1 = __ldg(sp + 1);
    float4 s2 = __ldg(sp + 2);
    depth = s2.y;
    if (__float_as_int(s2.z) <= 0) return false;
    return footprint_of(s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, f);
}

__global__ void bin_count_kernel(const dass_splat* __restrict__ splats, long long n_rec, CamTable ct,
                                 uint32_t* __restrict__ keys, uint32_t* __restrict__ counts) {
    long long rec = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (rec >= n_rec) return;
    const CamInfo& cam = ct.c[cam_of_record(ct, rec)];
    Footprint f;
    float depth;
    int cnt = 0;
    if (record_footprint(splats, rec, f, depth)) {
        int x0, x1, y0, y1;
        footprint_tiles(f, cam.tiles_x, cam.tiles_y, ct.tile, x0, x1, y0, y1);
        for (int y = y0; y <= y1; ++y) {
            int r0, r1;
            if (footprint_row(f, y, ct.tile, cam.tiles_x, r0, r1)) cnt += r1 - r0 + 1;
        }
    }
    keys[rec] = __float_as_uint(depth);     // positive depths: the bits order like the values
    counts[rec] = (uint32_t)cnt;
}

// Warp-wide inclusive sum of v (all lanes take part).
__device__ __forceinline__ uint32_t warp_inclusive_sum(uint32_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Emit the pairs of each record (record order) into its scanned slot range, each with its tile and
// its rank within the tile (an atomic per-tile counter; the order of the ranks is arbitrary, the
// per-tile sort restores the depth order). A warp owns 32
// consecutive records and the contiguous output range their pairs fill. The work is balanced
// over the lanes in three steps instead of each lane looping over its own record's tiles:
//   1. each lane computes its record's footprint and tile-row range; a warp scan numbers the
//      (record, tile row) units;
//   2. units are dealt to the lanes 32 at a time: a lane finds its unit's record (binary search
//      over the lanes' first unit), solves that tile row's run of tiles (the same footprint_row
//      that counted the pairs) and a warp scan gives the run's output offset;
//   3. output slots are dealt to the lanes in order: a lane finds its slot's unit (binary search
//      over the staged runs) and writes (tile, rank, record) -- consecutive lanes write consecutive
//      slots, and their tiles are mostly distinct, which spreads the counter atomics.
// A warp whose records have more than kDupUnits tile rows (very large footprints) writes its
// pairs lane by lane instead.
constexpr int kDupThreads = 256;
constexpr int kDupUnits = 128;
__global__ void __launch_bounds__(kDupThreads) duplicate_kernel(
    const dass_splat* __restrict__ splats, long long n_rec, CamTable ct, const uint32_t* __restrict__ offsets,
    const long long* total, long long capacity, uint32_t* __restrict__ pair_tile, uint32_t* __restrict__ pair_rank,
    uint32_t* __restrict__ pair_rec, uint32_t* __restrict__ tile_count, long long* counters) {
    constexpr int NW = kDupThreads / 32;
    __shared__ Footprint s_f[kDupThreads];
    __shared__ int s_y0[kDupThreads];
    __shared__ int s_cam[kDupThreads];
    __shared__ uint32_t s_upos[NW][kDupUnits];    // output offset of the unit's run (from the warp's base)
    __shared__ uint32_t s_utile[NW][kDupUnits];   // first tile of the run
    __shared__ uint32_t s_urec[NW][kDupUnits];
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long m = *total;
    if (k == 0) {
        counters[0] = m;
        counters[1] = m > capacity ? 1 : 0;
        counters[2] = m > capacity ? capacity : m;   // pairs actually stored (sort length)
    }
    const long long k0 = k - lane;
    if (k0 >= n_rec) return;                          // warp-uniform
    const bool active = k < n_rec;
    uint32_t rec = 0;
    long long pos = 0;
    if (active) {
        rec = (uint32_t)k;
        pos = offsets[k];
    }
    const long long wbase = __shfl_sync(0xffffffffu, pos, 0);
    const long long wend = k0 + 32 < n_rec ? (long long)offsets[k0 + 32] : m;
    // 1. footprint and tile rows of this lane's record
    Footprint f;
    float depth;
    int ci = 0, y0 = 0, y1 = -1;
    if (active && record_footprint(splats, rec, f, depth)) {
        ci = cam_of_record(ct, rec);
        const CamInfo& cam = ct.c[ci];
        int x0, x1;
        footprint_tiles(f, cam.tiles_x, cam.tiles_y, ct.tile, x0, x1, y0, y1);
    }
    const uint32_t nrows = y1 >= y0 ? (uint32_t)(y1 - y0 + 1) : 0u;
    const uint32_t rows_incl = warp_inclusive_sum(nrows, lane);
    const uint32_t ubase = rows_incl - nrows;
    const uint32_t U = __shfl_sync(0xffffffffu, rows_incl, 31);
    if (U > (uint32_t)kDupUnits) {                    // warp-uniform: lane-by-lane emission
        if (nrows) {
            const CamInfo& cam = ct.c[ci];
            for (int y = y0; y <= y1; ++y) {
                int r0, r1;
                if (!footprint_row(f, y, ct.tile, cam.tiles_x, r0, r1)) continue;
                for (int x = r0; x <= r1; ++x, ++pos)
                    if (pos < capacity && pos < wend) {
                        const uint32_t t = (uint32_t)(cam.tile_base + y * cam.tiles_x + x);
                        pair_tile[pos] = t;
                        pair_rank[pos] = atomicAdd(tile_count + t, 1u);
                        pair_rec[pos] = rec;
                    }
            }
        }
        return;
    }
    s_f[threadIdx.x] = f;
    s_y0[threadIdx.x] = y0;
    s_cam[threadIdx.x] = ci;
    __syncwarp();
    // 2. the tile runs of the units, 32 at a time, in (record, row) order
    uint32_t carry = 0;
    for (uint32_t u0 = 0; u0 < U; u0 += 32) {
        const uint32_t u = u0 + lane;
        int owner = 0;                                  // last lane whose first unit is <= u
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t b = __shfl_sync(0xffffffffu, ubase, owner + step);
            if (b <= u) owner += step;
        }
        const uint32_t orow = __shfl_sync(0xffffffffu, ubase, owner);
        const uint32_t orec = __shfl_sync(0xffffffffu, rec, owner);
        uint32_t len = 0, tile0 = 0;
        if (u < U) {
            const int src = (warp << 5) + owner;
            const CamInfo& cam = ct.c[s_cam[src]];
            const int y = s_y0[src] + (int)(u - orow);
            int r0, r1;
            if (footprint_row(s_f[src], y, ct.tile, cam.tiles_x, r0, r1)) {
                len = (uint32_t)(r1 - r0 + 1);
                tile0 = (uint32_t)(cam.tile_base + y * cam.tiles_x + r0);
            }
        }
        const uint32_t incl = warp_inclusive_sum(len, lane);
        if (u < U) {
            s_upos[warp][u] = carry + incl - len;
            s_utile[warp][u] = tile0;
            s_urec[warp][u] = orec;
        }
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncwarp();
    // 3. the pairs, slot by slot (the counted total bounds the warp's range)
    const long long span = wend - wbase;
    const uint32_t npairs = (long long)carry < span ? carry : (uint32_t)span;
    for (uint32_t i = lane; i < npairs; i += 32) {
        int lo = 0;                                     // last unit whose run starts at or before i
#pragma unroll
        for (int step = kDupUnits / 2; step > 0; step >>= 1) {
            const int c = lo + step;
            if (c < (int)U && s_upos[warp][c] <= i) lo = c;
        }
        const long long p = wbase + i;
        if (p < capacity) {
            const uint32_t t = s_utile[warp][lo] + (i - s_upos[warp][lo]);
            pair_tile[p] = t;
            pair_rank[p] = atomicAdd(tile_count + t, 1u);
            pair_rec[p] = s_urec[warp][lo];
        }
    }
}

// [start, end) of every tile's run from the scanned tile counts (0, 0 for an empty tile).
__global__ void tile_ranges_kernel(const uint32_t* __restrict__ start, const uint32_t* __restrict__ count, int tiles,
                                   uint32_t* __restrict__ ranges) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= tiles) return;
    const uint32_t c = count[t], s0 = c ? start[t] : 0u;
    ranges[2 * (long long)t] = s0;
    ranges[2 * (long long)t + 1] = s0 + c;
}

// Pair p goes to slot start[tile] + rank of its tile's range, as the key depth bits << 32 | record.
__global__ void bucket_scatter_kernel(const uint32_t* __restrict__ pair_tile, const uint32_t* __restrict__ pair_rank,
                                      const uint32_t* __restrict__ pair_rec, const uint32_t* __restrict__ depth_key,
                                      const uint32_t* __restrict__ tile_start, const long long* stored,
                                      unsigned long long* __restrict__ keys) {
    const long long n = *stored;
    const long long step = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += step) {
        const uint32_t r = pair_rec[p];
        keys[tile_start[pair_tile[p]] + pair_rank[p]] = ((unsigned long long)depth_key[r] << 32) | r;
    }
}

__device__ __forceinline__ void cmp_swap(unsigned long long& a, unsigned long long& b) {
    const unsigned long long lo = a < b ? a : b, hi = a < b ? b : a;
    a = lo;
    b = hi;
}

// Ascending bitonic sorting network over positions [0, n2) (n2 a power of two) of `s`, with every
// position >= len holding the largest key: for each block size k the first step compares position
// i with its mirror k - 1 - i inside the block, the next steps compare i with i + j for j = k/4 ..
// 1; every comparison puts the smaller key at the lower position, so the padding never moves below
// len and comparisons whose upper position is >= len can be skipped. One barrier per step.
// Comparison t of a step with distance j (j a power of two): positions lo = 2t - (t mod j) (the
// t-th position whose bit j is clear) and, for the mirror step of block size k = 2j, hi = lo xor
// (k - 1), else hi = lo + j. I is int for shared memory and long long in global memory.
template <int NT, class I, class Keys>
__device__ void bitonic_sort(Keys s, I len, I n2) {
    for (I k = 2; k <= n2; k <<= 1) {
        const I half = k >> 1;
        for (I t = threadIdx.x; t < n2 / 2; t += NT) {
            const I lo = 2 * t - (t & (half - 1)), hi = lo ^ (k - 1);
            if (hi < len) cmp_swap(s[lo], s[hi]);
        }
        __syncthreads();
        for (I j = k >> 2; j > 0; j >>= 1) {
            for (I t = threadIdx.x; t < n2 / 2; t += NT) {
                const I lo = 2 * t - (t & (j - 1)), hi = lo + j;
                if (hi < len) cmp_swap(s[lo], s[hi]);
            }
            __syncthreads();
        }
    }
}

__device__ __forceinline__ long long pow2_at_least(long long n) {
    long long p = 1;
    while (p < n) p <<= 1;
    return p;
}

// One CTA per tile: sort the tile's keys (depth bits << 32 | record) in shared memory and write
// the records. Lists longer than kSortCap are queued for big_tile_sort_kernel.
__global__ void __launch_bounds__(kSortThreads) tile_sort_kernel(const unsigned long long* __restrict__ keys,
                                                                 const uint32_t* __restrict__ ranges,
                                                                 uint32_t* __restrict__ pair_rec,
                                                                 uint32_t* __restrict__ big_list,
                                                                 unsigned int* __restrict__ big_count) {
    __shared__ unsigned long long s[kSortCap];
    const int tile = blockIdx.x;
    const uint32_t start = ranges[2 * (long long)tile];
    const int len = (int)(ranges[2 * (long long)tile + 1] - start);
    if (len <= 1) {
        if (len == 1 && threadIdx.x == 0) pair_rec[start] = (uint32_t)keys[start];
        return;
    }
    if (len > kSortCap) {
        if (threadIdx.x == 0) big_list[atomicAdd(big_count, 1u)] = (uint32_t)tile;
        return;
    }
    const int n2 = (int)pow2_at_least(len);
    for (int i = threadIdx.x; i < n2; i += kSortThreads) s[i] = i < len ? keys[start + i] : ~0ull;
    __syncthreads();
    bitonic_sort<kSortThreads, int>(s, len, n2);
    for (int i = threadIdx.x; i < len; i += kSortThreads) pair_rec[start + i] = (uint32_t)s[i];
}

// Tiles whose lists exceed kSortCap: up to kBigCap keys in dynamic shared memory, longer lists with
// the same network run in place on the keys in global memory (positions beyond the list are never
// touched). Persistent CTAs walk the queue.
__global__ void __launch_bounds__(kBigThreads) big_tile_sort_kernel(unsigned long long* __restrict__ keys,
                                                                    const uint32_t* __restrict__ ranges,
                                                                    uint32_t* __restrict__ pair_rec,
                                                                    const uint32_t* __restrict__ big_list,
                                                                    const unsigned int* __restrict__ big_count) {
    extern __shared__ unsigned long long sbig[];
    const unsigned int nb = *big_count;
    for (unsigned int b = blockIdx.x; b < nb; b += gridDim.x) {
        const long long tile = big_list[b];
        const uint32_t start = ranges[2 * tile];
        const long long len = (long long)(ranges[2 * tile + 1] - start);
        const long long n2 = pow2_at_least(len);
        if (len <= kBigCap) {
            for (int i = threadIdx.x; i < (int)n2; i += kBigThreads) sbig[i] = i < len ? keys[start + i] : ~0ull;
            __syncthreads();
            bitonic_sort<kBigThreads, int>(sbig, (int)len, (int)n2);
            for (int i = threadIdx.x; i < (int)len; i += kBigThreads) pair_rec[start + i] = (uint32_t)sbig[i];
        } else {
            bitonic_sort<kBigThreads, long long>(keys + start, len, n2);
            for (long long i = threadIdx.x; i < len; i += kBigThreads) pair_rec[start + i] = (uint32_t)keys[start + i];
        }
        __syncthreads();
    }
}

__global__ void set_len_kernel(long long* dst, long long v) { *dst = v; }

// ----------------------------------------------------------------- host-side orchestration

struct Carver {
    char* p;
    size_t used = 0;
    size_t cap;
    template <class T>
    T* take(long long count) {
        size_t bytes = ((size_t)count * sizeof(T) + 255) & ~(size_t)255;
        T* r = reinterpret_cast<T*>(p ? p + used : nullptr);
        used += bytes;
        return r;
    }
};

struct SortScratch {
    long long* scal;             // [8] device scalars: 0 n_rec, 1 tiles, 2 total pairs
    uint32_t* depth_key;         // record-sized
    uint32_t* counts;            // record-sized
    uint32_t* offsets;           // record-sized
    unsigned long long* partial; // scan partials
    uint32_t* tile_count;        // tile-sized
    uint32_t* tile_start;        // tile-sized
    uint32_t* big_list;          // tile-sized
    unsigned int* big_count;
    uint32_t* pair_tile;         // pair-sized
    uint32_t* pair_rank;
    uint32_t* pair_rec;
    unsigned long long* keys;    // pair-sized
};

SortScratch carve(Carver& cv, long long n_rec, long long cap, long long tiles) {
    SortScratch s;
    const long long scan_len = n_rec > tiles ? n_rec : tiles;
    s.scal = cv.take<long long>(8);
    s.depth_key = cv.take<uint32_t>(n_rec);
    s.counts = cv.take<uint32_t>(n_rec);
    s.offsets = cv.take<uint32_t>(n_rec);
    s.partial = cv.take<unsigned long long>(scan_len / kScanTile + 2);
    s.tile_count = cv.take<uint32_t>(tiles);
    s.tile_start = cv.take<uint32_t>(tiles);
    s.big_list = cv.take<uint32_t>(tiles);
    s.big_count = cv.take<unsigned int>(1);
    s.pair_tile = cv.take<uint32_t>(cap);
    s.pair_rank = cv.take<uint32_t>(cap);
    s.pair_rec = cv.take<uint32_t>(cap);
    s.keys = cv.take<unsigned long long>(cap);
    return s;
}

// out = exclusive_scan(in) over *len_dev elements (capacity len_cap); total -> *total (optional).
int scan_u32(const uint32_t* in, uint32_t* out, const long long* len_dev, long long len_cap,
             unsigned long long* partial, long long* total, cudaStream_t st) {
    int nb = div_up(len_cap > 0 ? len_cap : 1, kScanTile);
    scan_reduce_kernel<<<nb, kScanThreads, 0, st>>>(in, len_dev, partial); count_launch();
    scan_partials_kernel<<<1, 1024, 0, st>>>(partial, len_dev, total); count_launch();
    scan_down_kernel<<<nb, kScanThreads, 0, st>>>(in, out, len_dev, partial); count_launch();
    return check_launch("scan_u32");
}

}  // namespace

size_t bin_sort_workspace_bytes(long long n_rec, long long cap, long long tiles) {
    Carver cv{nullptr, 0, 0};
    carve(cv, n_rec, cap, tiles);
    return cv.used;
}

// Kernel attributes that must be set outside stream capture (the big-tile sort's shared memory).
int sort_prepare() {
    return allow_dynamic_smem(reinterpret_cast<const void*>(big_tile_sort_kernel),
                              kBigCap * (int)sizeof(unsigned long long));
}

int bin_sort_launch(const dass_splat* splats, long long n_rec, const CamTable& ct, uint32_t* pair_rec,
                    long long cap, uint32_t* tile_ranges, long long* counters, void* ws, size_t ws_bytes,
                    cudaStream_t st) {
    const long long tiles = ct.tiles_total;
    Carver cv{reinterpret_cast<char*>(ws), 0, ws_bytes};
    SortScratch s = carve(cv, n_rec, cap, tiles);
    if (cv.used > ws_bytes) return DASS_ERR_OOM;
    if (n_rec == 0 || tiles == 0) {
        DASS_CHECK_CUDA(cudaMemsetAsync(tile_ranges, 0, sizeof(uint32_t) * 2 * (size_t)tiles, st));
        DASS_CHECK_CUDA(cudaMemsetAsync(counters, 0, sizeof(long long) * 3, st));
        return DASS_OK;
    }
    if (int rc = sort_prepare()) return rc;
    DASS_CHECK_CUDA(cudaMemsetAsync(s.tile_count, 0, sizeof(uint32_t) * (size_t)tiles, st));
    DASS_CHECK_CUDA(cudaMemsetAsync(s.big_count, 0, sizeof(unsigned int), st));
    set_len_kernel<<<1, 1, 0, st>>>(s.scal + 0, n_rec); count_launch();
    set_len_kernel<<<1, 1, 0, st>>>(s.scal + 1, tiles); count_launch();
    // 1) tiles per record and the records' pair slots
    bin_count_kernel<<<div_up(n_rec, 256), 256, 0, st>>>(splats, n_rec, ct, s.depth_key, s.counts); count_launch();
    int rc = check_launch("bin_count");
    if (rc) return rc;
    rc = scan_u32(s.counts, s.offsets, s.scal + 0, n_rec, s.partial, s.scal + 2, st);
    if (rc) return rc;
    // 2) (tile, rank, record) per pair (stored count -> counters[2]), tile ranges, bucket scatter
    duplicate_kernel<<<div_up(n_rec, kDupThreads), kDupThreads, 0, st>>>(splats, n_rec, ct, s.offsets, s.scal + 2,
                                                                         cap, s.pair_tile, s.pair_rank, s.pair_rec,
                                                                         s.tile_count, counters);
    count_launch();
    if ((rc = check_launch("duplicate"))) return rc;
    rc = scan_u32(s.tile_count, s.tile_start, s.scal + 1, tiles, s.partial, nullptr, st);
    if (rc) return rc;
    tile_ranges_kernel<<<div_up(tiles, 256), 256, 0, st>>>(s.tile_start, s.tile_count, (int)tiles, tile_ranges);
    count_launch();
    const int sb = div_up(cap > 0 ? cap : 1, 256);
    bucket_scatter_kernel<<<sb < 152 * 16 ? sb : 152 * 16, 256, 0, st>>>(s.pair_tile, s.pair_rank, s.pair_rec,
                                                                         s.depth_key, s.tile_start, counters + 2,
                                                                         s.keys);
    count_launch();
    if ((rc = check_launch("bucket_scatter"))) return rc;
    // 3) per-tile sort by (depth, record)
    tile_sort_kernel<<<(int)tiles, kSortThreads, 0, st>>>(s.keys, tile_ranges, pair_rec, s.big_list, s.big_count);
    count_launch();
    big_tile_sort_kernel<<<kBigBlocks, kBigThreads, kBigCap * sizeof(unsigned long long), st>>>(
        s.keys, tile_ranges, pair_rec, s.big_list, s.big_count);
    count_launch();
    return check_launch("tile_sort");
}

// Generic pieces reused by other translation units.
size_t scan_partials_bytes(long long len) { return sizeof(unsigned long long) * (size_t)(len / kScanTile + 2); }

int scan_u32_public(const uint32_t* in, uint32_t* out, const long long* len_dev, long long len_cap,
                    unsigned long long* partial, long long* total, cudaStream_t st) {
    return scan_u32(in, out, len_dev, len_cap, partial, total, st);
}

}  // namespace dass
