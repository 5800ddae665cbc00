// Tile binning and a hand-written stable LSD radix sort (no CUB) for the tile-based
// rasteriser. The pair order is that of the 64-bit key (tile id << 32 | depth bits), ties in
// record order: the 32 depth-bit digits are sorted on the records before duplication (all
// pairs of a record share its depth), the tile-id digits on the pairs afterwards.
//
// Every kernel reads its item count from device memory and sizes its work from it, so the
// whole sequence needs no host synchronisation and can be captured in a CUDA graph; grids are
// launched for the capacity and surplus blocks exit at once.
#include "launch.cuh"

namespace dass {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;   // 2048 elements per scan block

constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 16;
constexpr int kRadixTile = kRadixThreads * kRadixItems;  // 4096 keys per radix block
constexpr int kMaxDigitBits = 9;
constexpr int kMaxDigits = 1 << kMaxDigitBits;
constexpr int kRadixWarps = kRadixThreads / 32;

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

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

// ----------------------------------------------------------------- radix sort passes

__device__ __forceinline__ long long radix_nblocks(long long n) { return (n + kRadixTile - 1) / kRadixTile; }

// Per-block digit counts, digit-major: hist[d * nb + b].
__global__ void __launch_bounds__(kRadixThreads) radix_hist_kernel(const uint32_t* __restrict__ keys,
                                                                   const long long* n_dev, uint32_t* __restrict__ hist,
                                                                   long long* hist_len, int shift, int dbits) {
    long long n = *n_dev;
    long long nb = radix_nblocks(n);
    int nd = 1 << dbits;
    if (blockIdx.x == 0 && threadIdx.x == 0) *hist_len = nb * nd;
    if ((long long)blockIdx.x >= nb) return;
    __shared__ uint32_t sh[kMaxDigits];
    for (int d = threadIdx.x; d < nd; d += kRadixThreads) sh[d] = 0;
    __syncthreads();
    unsigned mask = (unsigned)nd - 1u;
    long long base = (long long)blockIdx.x * kRadixTile;
    // all loads of the block are issued before any is used (one memory latency per block)
    uint32_t kr[kRadixItems];
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        long long idx = base + r * kRadixThreads + threadIdx.x;
        kr[r] = idx < n ? keys[idx] : 0u;
    }
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        long long idx = base + r * kRadixThreads + threadIdx.x;
        if (idx < n) atomicAdd(&sh[(kr[r] >> shift) & mask], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < nd; d += kRadixThreads) hist[(long long)d * nb + blockIdx.x] = sh[d];
}

// Lanes of `among` whose digit equals this lane's (one ballot per digit bit; the cost does not
// grow with the number of distinct digits in the warp).
__device__ __forceinline__ unsigned digit_peers(unsigned digit, int dbits, unsigned among) {
    unsigned peers = among;
#pragma unroll
    for (int b = 0; b < kMaxDigitBits; ++b) {
        if (b < dbits) {
            const bool bit = (digit >> b) & 1u;
            const unsigned bal = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? bal : ~bal;
        }
    }
    return peers;
}

// Block-wide exclusive scan of v over the 256 threads (one value each); returns the prefix.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* s_warp) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    uint32_t woff = 0;
#pragma unroll
    for (int w = 0; w < kRadixWarps; ++w) woff += w < warp ? s_warp[w] : 0u;
    return woff + incl - v;
}

// Stable scatter of one pass. Warp w owns the contiguous keys [w*kRadixItems*32, (w+1)*...) of
// the block's tile (blocked arrangement: warp, then round, then lane is key order). A key's
// rank among equal digits is its warp's running count (ballot-based peer masks per round) plus the counts of
// the warps before it; a block-wide scan over digits gives each key its slot in a block-local
// digit-sorted order. Keys and values are exchanged through shared memory into that order and
// written out so that consecutive threads write consecutive positions of each digit's output
// run (coalesced), at the block's scanned global digit offsets.
__global__ void __launch_bounds__(kRadixThreads) radix_scatter_kernel(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in, uint32_t* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out, const long long* n_dev, const uint32_t* __restrict__ hist_scanned, int shift,
    int dbits) {
    const long long n = *n_dev;
    const long long nb = radix_nblocks(n);
    if ((long long)blockIdx.x >= nb) return;
    const int nd = 1 << dbits;
    const unsigned mask = (unsigned)nd - 1u;
    constexpr int kWarpItems = kRadixItems * 32;
    // s_cnt (per-warp digit counts, then per-warp offsets) and later the exchanged keys/values
    // share one buffer: the counts are dead once every key knows its local slot.
    __shared__ uint32_t s_buf[2 * kRadixTile];
    __shared__ uint32_t s_start[kMaxDigits];    // block-local start of each digit
    __shared__ uint32_t s_gbase[kMaxDigits];    // global output start of each digit (this block)
    __shared__ uint32_t s_warp[kRadixWarps];
    uint32_t(*s_cnt)[kMaxDigits] = reinterpret_cast<uint32_t(*)[kMaxDigits]>(s_buf);
    uint32_t* s_key = s_buf;
    uint32_t* s_val = s_buf + kRadixTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long tile0 = (long long)blockIdx.x * kRadixTile;
    const long long base = tile0 + (long long)warp * kWarpItems;
    // the block's keys and values are requested first, so the global latency of the (strided)
    // digit offsets below overlaps with them
    uint32_t kr[kRadixItems], vr[kRadixItems], slot[kRadixItems];
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        const long long idx = base + r * 32 + lane;
        kr[r] = idx < n ? __ldcs(keys_in + idx) : 0u;
        vr[r] = idx < n ? __ldcs(vals_in + idx) : 0u;
    }
    for (int d = threadIdx.x; d < nd; d += kRadixThreads) {
        s_gbase[d] = hist_scanned[(long long)d * nb + blockIdx.x];
#pragma unroll
        for (int w = 0; w < kRadixWarps; ++w) s_cnt[w][d] = 0;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        const bool valid = base + r * 32 + lane < n;
        const unsigned digit = (kr[r] >> shift) & mask;
        const unsigned peers = digit_peers(digit, dbits, __ballot_sync(0xffffffffu, valid));
        const uint32_t before = valid ? s_cnt[warp][digit] : 0u;
        slot[r] = before + (uint32_t)__popc(peers & lanemask_lt());
        __syncwarp();
        if (valid && (__ffs(peers) - 1) == lane) s_cnt[warp][digit] = before + (uint32_t)__popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: warp offsets within the digit and the digit's total; 2 digits per thread
    uint32_t tot = 0;
    for (int d = 2 * threadIdx.x; d < 2 * threadIdx.x + 2 && d < nd; ++d) {
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kRadixWarps; ++w) {
            const uint32_t c = s_cnt[w][d];
            s_cnt[w][d] = run;
            run += c;
        }
        s_start[d] = run;     // digit total for now
        tot += run;
    }
    const uint32_t pre = block_exclusive_scan(tot, s_warp);
    if (2 * threadIdx.x < nd) {
        const uint32_t t0 = s_start[2 * threadIdx.x];
        s_start[2 * threadIdx.x] = pre;
        if (2 * threadIdx.x + 1 < nd) s_start[2 * threadIdx.x + 1] = pre + t0;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        const bool valid = base + r * 32 + lane < n;
        const unsigned digit = (kr[r] >> shift) & mask;
        if (valid) slot[r] += s_start[digit] + s_cnt[warp][digit];
    }
    __syncthreads();    // counts are dead from here on: the buffer takes the keys and values
#pragma unroll
    for (int r = 0; r < kRadixItems; ++r) {
        if (base + r * 32 + lane < n) {
            s_key[slot[r]] = kr[r];
            s_val[slot[r]] = vr[r];
        }
    }
    __syncthreads();
    const int cnt = (int)(n - tile0 < kRadixTile ? n - tile0 : kRadixTile);
    for (int i = threadIdx.x; i < cnt; i += kRadixThreads) {
        const uint32_t key = s_key[i];
        const unsigned digit = (key >> shift) & mask;
        const uint32_t pos = s_gbase[digit] + (uint32_t)i - s_start[digit];
        keys_out[pos] = key;
        vals_out[pos] = s_val[i];
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

// Item i is record list[i] (list null: record i), i < *n_dev. A record whose row (its index within
// its camera's segment) is flagged in skip_rows emits no pairs, like a culled one.
__global__ void bin_count_kernel(const dass_splat* __restrict__ splats, const long long* __restrict__ n_dev,
                                 const uint32_t* __restrict__ list, const uint8_t* __restrict__ skip_rows, CamTable ct,
                                 uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                 uint32_t* __restrict__ counts) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *n_dev) return;
    const long long rec = list ? (long long)list[i] : i;
    const CamInfo& cam = ct.c[cam_of_record(ct, rec)];
    Footprint f;
    float depth;
    int cnt = 0;
    if (!(skip_rows && skip_rows[rec - cam.rec_base]) && record_footprint(splats, rec, f, depth)) {
        int x0, x1, y0, y1;
        footprint_tiles(f, cam.tiles_x, cam.tiles_y, ct.tile, x0, x1, y0, y1);
        for (int y = y0; y <= y1; ++y) {
            int r0, r1;
            if (footprint_row(f, y, ct.tile, cam.tiles_x, r0, r1)) cnt += r1 - r0 + 1;
        }
    }
    keys[i] = cnt > 0 ? __float_as_uint(depth) : 0xffffffffu;
    vals[i] = (uint32_t)i;
    counts[i] = (uint32_t)cnt;
}

// out[i] = counts[order[i]], and rec[i] = list[order[i]] when there is a list (else the record ids in
// depth order are order itself): the pair counts and record ids in depth order.
__global__ void gather_counts_kernel(const uint32_t* __restrict__ order, const uint32_t* __restrict__ counts,
                                     const uint32_t* __restrict__ list, uint32_t* __restrict__ out,
                                     uint32_t* __restrict__ rec, const long long* __restrict__ n_dev) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= *n_dev) return;
    const uint32_t o = order[i];
    out[i] = counts[o];
    if (list) rec[i] = list[o];
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

// Emit the pairs of each record (depth order) into its scanned slot range. A warp owns 32
// consecutive records and the contiguous output range their pairs fill. The work is balanced
// over the lanes in three steps instead of each lane looping over its own record's tiles:
//   1. each lane computes its record's footprint and tile-row range; a warp scan numbers the
//      (record, tile row) units;
//   2. units are dealt to the lanes 32 at a time: a lane finds its unit's record (binary search
//      over the lanes' first unit), solves that tile row's run of tiles (the same footprint_row
//      that counted the pairs) and a warp scan gives the run's output offset;
//   3. output slots are dealt to the lanes in order: a lane finds its slot's unit (binary search
//      over the staged runs) and writes (tile, record) -- consecutive lanes write consecutive
//      slots.
// A warp whose records have more than kDupUnits tile rows (very large footprints) writes its
// pairs lane by lane instead.
constexpr int kDupThreads = 256;
constexpr int kDupUnits = 128;
__global__ void __launch_bounds__(kDupThreads) duplicate_kernel(
    const dass_splat* __restrict__ splats, const long long* __restrict__ n_dev, CamTable ct,
    const uint32_t* __restrict__ order, const uint32_t* __restrict__ offsets, const long long* total,
    long long capacity, uint32_t* __restrict__ pair_tile, uint32_t* __restrict__ pair_rec, long long* counters) {
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
    const long long n_rec = *n_dev;
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
        rec = order[k];
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
                        pair_tile[pos] = (uint32_t)(cam.tile_base + y * cam.tiles_x + x);
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
            pair_tile[p] = s_utile[warp][lo] + (i - s_upos[warp][lo]);
            pair_rec[p] = s_urec[warp][lo];
        }
    }
}

// [start, end) of every tile's run in the sorted pair list. Grid-stride over groups of 4
// consecutive pairs: one 16-byte load per group (the key buffer is 256-byte aligned and its
// capacity a multiple of 64 keys, so the group never leaves the buffer; keys at or beyond n are
// ignored) plus the keys just before and after it.
__global__ void tile_ranges_kernel(const uint32_t* __restrict__ tiles, const long long* n_dev,
                                   uint32_t* __restrict__ ranges) {
    const long long n = *n_dev;
    const long long nq = (n + 3) / 4;
    const long long step = (long long)gridDim.x * blockDim.x;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += step) {
        const long long i0 = 4 * q;
        const uint4 v = __ldcs(reinterpret_cast<const uint4*>(tiles + i0));
        const uint32_t t[4] = {v.x, v.y, v.z, v.w};
        uint32_t prev = i0 > 0 ? __ldg(tiles + i0 - 1) : 0xffffffffu;
        const uint32_t after = i0 + 4 < n ? __ldg(tiles + i0 + 4) : 0xffffffffu;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const long long i = i0 + k;
            if (i >= n) break;
            const uint32_t next = k < 3 ? (i + 1 < n ? t[k + 1] : 0xffffffffu) : after;
            if (i == 0 || prev != t[k]) ranges[2 * (long long)t[k]] = (uint32_t)i;
            if (next != t[k]) ranges[2 * (long long)t[k] + 1] = (uint32_t)(i + 1);
            prev = t[k];
        }
    }
}

__global__ void set_len_kernel(long long* dst, long long v) { *dst = v; }

// ----------------------------------------------------------------- incremental binning
// A stage trains a subset of the Gaussians (the dynamic rows in the shift stage, the var rows in
// the inheritance and densification stages); the records of the other rows do not change over the
// stage's iterations. Their pairs are binned and sorted once (the static lists, with each pair's
// depth key and each tile's first position), and every iteration bins and sorts only the moving
// rows' records and merges the two lists tile by tile: the result is the full binning's, pair for
// pair, because both orders are the one of the key (tile, depth bits, record id).

// First index of the sorted keys [0, n) that is >= v.
__device__ __forceinline__ long long lower_bound_u32(const uint32_t* __restrict__ keys, long long n, uint32_t v) {
    long long lo = 0, hi = n;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (__ldg(keys + mid) < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// start[t] = first sorted position of tile t (t = 0 .. tiles_total; start[tiles_total] = stored count).
__global__ void tile_start_kernel(const uint32_t* __restrict__ keys, const long long* __restrict__ n_dev,
                                  int tiles_total, uint32_t* __restrict__ start) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t > tiles_total) return;
    start[t] = (uint32_t)lower_bound_u32(keys, *n_dev, (uint32_t)t);
}

// depth[i] = the sort key (depth bits) of the record of pair i, i < *n_dev.
__global__ void pair_depth_kernel(const dass_splat* __restrict__ splats, const uint32_t* __restrict__ rec,
                                  const long long* __restrict__ n_dev, uint32_t* __restrict__ depth) {
    const long long n = *n_dev;
    const long long step = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += step)
        depth[i] = __float_as_uint(__ldg(&splats[rec[i]].depth));
}

// Records of the moving rows, camera-major and ascending: list[c m + k] = rec_base(c) + rows[k] for the
// m = *m_dev rows (ascending); *n_list = n_cams m.
__global__ void moving_list_kernel(const int* __restrict__ rows, const long long* __restrict__ m_dev, CamTable ct,
                                   uint32_t* __restrict__ list, long long* __restrict__ n_list) {
    const long long m = *m_dev;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *n_list = m * ct.n;
    if (i >= m * ct.n) return;
    const long long c = i / m, k = i - c * m;
    list[i] = (uint32_t)(ct.c[c].rec_base + rows[k]);
}

// *dst = min(*src, cap).
__global__ void copy_len_kernel(long long* __restrict__ dst, const long long* __restrict__ src, long long cap) {
    const long long v = *src;
    *dst = v < cap ? v : cap;
}

// One warp per tile: the tile's static pairs [s_start[t], s_start[t + 1]) and moving pairs
// [d_start[t], d_start[t + 1]) are merged by (depth bits, record id) into out_rec from the tile's
// first position, the static count of earlier tiles plus the moving count of earlier tiles. Keys are
// distinct (record ids are). The warp takes the static list in blocks of kMergeBlock keys staged in
// shared memory. The moving pairs below the block's last key (all remaining ones at the last block)
// are taken 32 at a time, one per lane: a binary search over the staged block gives the number p of
// static keys below it, so it goes to its own index plus the static pairs before the block plus p,
// and it adds one to the block's insertion count at p. A static key k of the block is then above
// the moving pairs of earlier blocks and above those of this block with p <= k (an inclusive scan of
// the insertion counts). Positions at or beyond cap are dropped and the ranges clamped to cap (the
// counters flag the overflow, as in the full binning); empty tiles get the range (0, 0).
constexpr int kMergeWarps = 8;
constexpr int kMergeBlock = 256;     // static keys staged per step
__global__ void __launch_bounds__(32 * kMergeWarps) merge_pairs_kernel(
    int tiles_total, const uint32_t* __restrict__ s_rec, const uint32_t* __restrict__ s_depth,
    const uint32_t* __restrict__ s_start, const long long* __restrict__ s_counters,
    const uint32_t* __restrict__ d_rec, const uint32_t* __restrict__ d_depth, const uint32_t* __restrict__ d_start,
    const long long* __restrict__ d_counters, long long cap, uint32_t* __restrict__ out_rec,
    uint32_t* __restrict__ ranges, long long* __restrict__ counters) {
    constexpr int B = kMergeBlock, PER = B / 32;
    constexpr int BC = B + B / 32 + 1;     // insertion counts, one pad word per 32 (conflict-free scan)
    __shared__ uint32_t sh_d[kMergeWarps][B];
    __shared__ uint32_t sh_r[kMergeWarps][B];
    __shared__ uint32_t sh_c[kMergeWarps][BC];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long t = (long long)blockIdx.x * kMergeWarps + w;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const long long total = s_counters[0] + d_counters[0];
        counters[0] = total;
        counters[1] = total > cap ? 1 : 0;
        counters[2] = total > cap ? cap : total;
    }
    if (t >= tiles_total) return;
    const uint32_t ss = s_start[t], se = s_start[t + 1], ds = d_start[t], de = d_start[t + 1];
    const long long base = (long long)ss + ds;
    const long long total = (long long)(se - ss) + (de - ds);
    if (lane == 0) {
        const long long b0 = base < cap ? base : cap, b1 = base + total < cap ? base + total : cap;
        ranges[2 * t] = total > 0 ? (uint32_t)b0 : 0u;
        ranges[2 * t + 1] = total > 0 ? (uint32_t)b1 : 0u;
    }
    if (total == 0) return;
    uint32_t* kd = sh_d[w];
    uint32_t* kr = sh_r[w];
    uint32_t* cnt = sh_c[w];
    auto cix = [](uint32_t k) { return k + (k >> 5); };   // padded index of insertion count k
    uint32_t q = ds;                  // next moving pair to place
    // the static block in flight: its keys are requested one block ahead
    uint32_t nd_[PER], nr_[PER];
#pragma unroll
    for (int m = 0; m < PER; ++m) {
        const uint32_t k = lane + 32 * m;
        nd_[m] = ss + k < se ? __ldg(s_depth + ss + k) : 0xffffffffu;
        nr_[m] = ss + k < se ? __ldg(s_rec + ss + k) : 0xffffffffu;
    }
    for (uint32_t g0 = ss; g0 < se; g0 += B) {
        const uint32_t nS = se - g0 < (uint32_t)B ? se - g0 : (uint32_t)B;
        const bool last_block = g0 + B >= se;
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const uint32_t k = lane + 32 * m;
            kd[k] = nd_[m];
            kr[k] = nr_[m];
            cnt[cix(k)] = 0u;
        }
        if (lane == 0) cnt[cix(B)] = 0u;
        if (!last_block) {
#pragma unroll
            for (int m = 0; m < PER; ++m) {
                const uint32_t k = g0 + B + lane + 32 * m;
                nd_[m] = k < se ? __ldg(s_depth + k) : 0xffffffffu;
                nr_[m] = k < se ? __ldg(s_rec + k) : 0xffffffffu;
            }
        }
        __syncwarp();
        const uint32_t ld = kd[nS - 1], lr = kr[nS - 1];
        const uint32_t q0 = q;
        while (q < de) {
            const uint32_t j = q + lane;
            const bool valid = j < de;
            const uint32_t dd = valid ? __ldg(d_depth + j) : 0xffffffffu;
            const uint32_t dr = valid ? __ldg(d_rec + j) : 0xffffffffu;
            const bool in_block = valid && (last_block || dd < ld || (dd == ld && dr < lr));
            const unsigned bal = __ballot_sync(0xffffffffu, in_block);    // a prefix of the lanes
            if (in_block) {
                uint32_t lo = 0, hi = nS;            // static keys of the block below (dd, dr)
                while (lo < hi) {
                    const uint32_t mid = (lo + hi) >> 1;
                    const uint32_t md = kd[mid];
                    if (md < dd || (md == dd && kr[mid] < dr)) lo = mid + 1;
                    else hi = mid;
                }
                const long long pos = base + (j - ds) + (g0 - ss) + lo;
                if (pos < cap) out_rec[pos] = dr;
                atomicAdd(&cnt[cix(lo)], 1u);
            }
            const uint32_t n_in = (uint32_t)__popc(bal);
            q += n_in;
            if (n_in < 32u) break;
        }
        __syncwarp();
        // inclusive scan of the insertion counts: lane l owns keys [PER l, PER l + PER)
        uint32_t v[PER];
        uint32_t run = 0;
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            run += cnt[cix(PER * lane + m)];
            v[m] = run;
        }
        uint32_t incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t excl = incl - run;
        __syncwarp();
#pragma unroll
        for (int m = 0; m < PER; ++m) cnt[cix(PER * lane + m)] = excl + v[m];
        __syncwarp();
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const uint32_t k = lane + 32 * m;
            if (k < nS) {
                const long long pos = base + (g0 - ss) + k + (q0 - ds) + cnt[cix(k)];
                if (pos < cap) out_rec[pos] = kr[k];
            }
        }
        __syncwarp();
    }
    // moving pairs above every static pair (all of them when the tile has no static pair)
    for (uint32_t j = q + lane; j < de; j += 32) {
        const long long pos = base + (j - ds) + (se - ss);
        if (pos < cap) out_rec[pos] = __ldg(d_rec + j);
    }
}

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
    long long* scal;             // [8] device scalars: 0 n_rec, 1 hist_len, 2 total pairs, 3.. spare
    uint32_t* kA; uint32_t* vA; uint32_t* kB; uint32_t* vB;   // record-sized
    uint32_t* counts;            // record-sized
    uint32_t* offsets;           // record-sized
    uint32_t* hist;              // digits * max blocks
    unsigned long long* partial; // scan partials
    uint32_t* pk0; uint32_t* pk1; uint32_t* pv1;  // pair-sized
};

long long hist_capacity(long long n_max) {
    return (long long)kMaxDigits * ((n_max + kRadixTile - 1) / kRadixTile + 1);
}

SortScratch carve(Carver& cv, long long n_rec, long long cap) {
    SortScratch s;
    long long big = n_rec > cap ? n_rec : cap;
    s.scal = cv.take<long long>(8);
    s.kA = cv.take<uint32_t>(n_rec);
    s.vA = cv.take<uint32_t>(n_rec);
    s.kB = cv.take<uint32_t>(n_rec);
    s.vB = cv.take<uint32_t>(n_rec);
    s.counts = cv.take<uint32_t>(n_rec);
    s.offsets = cv.take<uint32_t>(n_rec);
    s.hist = cv.take<uint32_t>(hist_capacity(big));
    long long scan_len = hist_capacity(big) > n_rec ? hist_capacity(big) : n_rec;
    s.partial = cv.take<unsigned long long>(scan_len / kScanTile + 2);
    s.pk0 = cv.take<uint32_t>(cap);
    s.pk1 = cv.take<uint32_t>(cap);
    s.pv1 = cv.take<uint32_t>(cap);
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

// Stable sort of (keys, vals) by bits [0, bits) of the keys; n from *n_dev (<= n_cap).
// Pass i reads buffer set i%2 and writes set (i+1)%2 of {(k0, v0), (k1, v1)}; returns the
// index of the set holding the result.
int radix_sort(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, const long long* n_dev, long long n_cap,
               int bits, SortScratch& s, cudaStream_t st, int* result_set) {
    int passes = (bits + kMaxDigitBits - 1) / kMaxDigitBits;
    if (passes < 1) passes = 1;
    int dbits = (bits + passes - 1) / passes;
    int nb = div_up(n_cap > 0 ? n_cap : 1, kRadixTile);
    long long hist_cap = (long long)(1 << dbits) * nb;
    uint32_t* kin = k0; uint32_t* vin = v0; uint32_t* kout = k1; uint32_t* vout = v1;
    for (int p = 0; p < passes; ++p) {
        int shift = p * dbits;
        int db = dbits;
        if (shift + db > bits) db = bits - shift;
        radix_hist_kernel<<<nb, kRadixThreads, 0, st>>>(kin, n_dev, s.hist, s.scal + 1, shift, db); count_launch();
        int rc = scan_u32(s.hist, s.hist, s.scal + 1, hist_cap, s.partial, nullptr, st);
        if (rc) return rc;
        radix_scatter_kernel<<<nb, kRadixThreads, 0, st>>>(kin, vin, kout, vout, n_dev, s.hist, shift, db); count_launch();
        int lc = check_launch("radix_pass");
        if (lc) return lc;
        uint32_t* tk = kin; kin = kout; kout = tk;
        uint32_t* tv = vin; vin = vout; vout = tv;
    }
    *result_set = passes % 2;
    return DASS_OK;
}

int bits_for(long long values) {
    int b = 1;
    while ((1ll << b) < values) ++b;
    return b;
}

}  // namespace

size_t bin_sort_workspace_bytes(long long n_rec, long long cap) {
    Carver cv{nullptr, 0, 0};
    carve(cv, n_rec, cap);
    return cv.used;
}

// Binning and sort of the items i < *s.scal (capacity n_cap; item i is record list[i], or record i
// when list is null; rows flagged in skip_rows emit nothing) into pair_rec[cap] and counters[3];
// *keys_out points at the sorted tile keys (workspace) on return.
int bin_sort_core(const dass_splat* splats, long long n_cap, const uint32_t* list, const uint8_t* skip_rows,
                  const CamTable& ct, uint32_t* pair_rec, long long cap, long long* counters, SortScratch& s,
                  cudaStream_t st, uint32_t** keys_out) {
    const long long* n_dev = s.scal + 0;
    bin_count_kernel<<<div_up(n_cap, 256), 256, 0, st>>>(splats, n_dev, list, skip_rows, ct, s.kA, s.vA, s.counts);
    count_launch();
    int rc = check_launch("bin_count");
    if (rc) return rc;
    // 1) depth digits on the records (32 bits)
    int set = 0;
    rc = radix_sort(s.kA, s.vA, s.kB, s.vB, n_dev, n_cap, 32, s, st, &set);
    if (rc) return rc;
    uint32_t* order = set == 0 ? s.vA : s.vB;
    uint32_t* recs = list ? (set == 0 ? s.vB : s.vA) : order;   // the other value buffer is free now
    // 2) pair offsets and record ids in depth order
    gather_counts_kernel<<<div_up(n_cap, 256), 256, 0, st>>>(order, s.counts, list, s.offsets, recs, n_dev);
    count_launch();
    rc = scan_u32(s.offsets, s.offsets, n_dev, n_cap, s.partial, s.scal + 2, st);
    if (rc) return rc;
    // 3) duplicate into tile-keyed pairs (stored count -> counters[2])
    int tbits = bits_for(ct.tiles_total > 1 ? ct.tiles_total : 2);
    int passes = (tbits + kMaxDigitBits - 1) / kMaxDigitBits;
    // the sort must end in (pk?, pair_rec): pass i writes set (i+1)%2; choose the start set
    uint32_t *k_out = s.pk0, *v_out = pair_rec, *k_tmp = s.pk1, *v_tmp = s.pv1;
    uint32_t *k_start = (passes % 2 == 0) ? k_out : k_tmp;
    uint32_t *v_start = (passes % 2 == 0) ? v_out : v_tmp;
    duplicate_kernel<<<div_up(n_cap, kDupThreads), kDupThreads, 0, st>>>(splats, n_dev, ct, recs, s.offsets,
                                                                         s.scal + 2, cap, k_start, v_start, counters);
    count_launch();
    rc = check_launch("duplicate");
    if (rc) return rc;
    // 4) tile digits on the pairs
    const long long* m_dev = counters + 2;
    if (passes % 2 == 0)
        rc = radix_sort(k_out, v_out, k_tmp, v_tmp, m_dev, cap, tbits, s, st, &set);
    else
        rc = radix_sort(k_tmp, v_tmp, k_out, v_out, m_dev, cap, tbits, s, st, &set);
    if (rc) return rc;
    *keys_out = k_out;
    return DASS_OK;
}

int bin_sort_launch(const dass_splat* splats, long long n_rec, const CamTable& ct, uint32_t* pair_rec,
                    long long cap, uint32_t* tile_ranges, long long* counters, void* ws, size_t ws_bytes,
                    cudaStream_t st) {
    Carver cv{reinterpret_cast<char*>(ws), 0, ws_bytes};
    SortScratch s = carve(cv, n_rec, cap);
    if (cv.used > ws_bytes) return DASS_ERR_OOM;
    DASS_CHECK_CUDA(cudaMemsetAsync(tile_ranges, 0, sizeof(uint32_t) * 2 * (size_t)ct.tiles_total, st));
    if (n_rec == 0) {
        DASS_CHECK_CUDA(cudaMemsetAsync(counters, 0, sizeof(long long) * 3, st));
        return DASS_OK;
    }
    set_len_kernel<<<1, 1, 0, st>>>(s.scal + 0, n_rec); count_launch();
    uint32_t* keys = nullptr;
    int rc = bin_sort_core(splats, n_rec, nullptr, nullptr, ct, pair_rec, cap, counters, s, st, &keys);
    if (rc) return rc;
    // 5) tile ranges
    const int rq = div_up(div_up(cap, 4), 256);
    tile_ranges_kernel<<<rq < 152 * 8 ? rq : 152 * 8, 256, 0, st>>>(keys, counters + 2, tile_ranges);
    count_launch();
    return check_launch("tile_ranges");
}

size_t bin_sort_split_workspace_bytes(long long n_rows, long long n_rec, long long cap) {
    const size_t a = bin_sort_workspace_bytes(n_rec, cap), b = mask_rows_workspace_bytes(n_rows);
    return a > b ? a : b;
}

int bin_sort_split_launch(const dass_splat* splats, long long n_rows, const CamTable& ct, const uint8_t* moving_rows,
                          long long cap, const StaticBins& sb, void* ws, size_t ws_bytes, cudaStream_t st) {
    const long long n_rec = (long long)ct.n * n_rows;
    if (n_rows <= 0 || ws_bytes < bin_sort_split_workspace_bytes(n_rows, n_rec, cap)) return DASS_ERR_OOM;
    // the moving rows (ascending), then their records camera by camera
    int rc = mask_rows_launch(moving_rows, n_rows, sb.rows, sb.n_rows_moving, ws, ws_bytes, st);
    if (rc) return rc;
    moving_list_kernel<<<div_up(n_rec, 256), 256, 0, st>>>(sb.rows, sb.n_rows_moving, ct, sb.moving, sb.n_moving);
    count_launch();
    if ((rc = check_launch("moving_list_kernel"))) return rc;
    // the static pairs: every record but the moving rows'
    Carver cv{reinterpret_cast<char*>(ws), 0, ws_bytes};
    SortScratch s = carve(cv, n_rec, cap);
    set_len_kernel<<<1, 1, 0, st>>>(s.scal + 0, n_rec); count_launch();
    uint32_t* keys = nullptr;
    if ((rc = bin_sort_core(splats, n_rec, nullptr, moving_rows, ct, sb.rec, cap, sb.counters, s, st, &keys)))
        return rc;
    tile_start_kernel<<<div_up(ct.tiles_total + 1, 256), 256, 0, st>>>(keys, sb.counters + 2, ct.tiles_total,
                                                                       sb.start);
    count_launch();
    pair_depth_kernel<<<152 * 8, 256, 0, st>>>(splats, sb.rec, sb.counters + 2, sb.depth);
    count_launch();
    return check_launch("bin_sort_split");
}

namespace {
struct MergeScratch {
    SortScratch s;
    uint32_t* rec;
    uint32_t* depth;
    uint32_t* start;
    long long* counters;
};
MergeScratch carve_merge(Carver& cv, long long moving_cap, long long cap, int tiles_total) {
    MergeScratch m;
    m.s = carve(cv, moving_cap, cap);
    m.rec = cv.take<uint32_t>(cap);
    m.depth = cv.take<uint32_t>(cap);
    m.start = cv.take<uint32_t>((long long)tiles_total + 1);
    m.counters = cv.take<long long>(4);
    return m;
}
}  // namespace

size_t bin_sort_merge_workspace_bytes(long long moving_cap, long long cap, int tiles_total) {
    Carver cv{nullptr, 0, 0};
    carve_merge(cv, moving_cap > 0 ? moving_cap : 1, cap, tiles_total);
    return cv.used;
}

int bin_sort_merge_launch(const dass_splat* splats, const CamTable& ct, const StaticBins& sb, long long moving_cap,
                          long long cap, uint32_t* pair_rec, uint32_t* tile_ranges, long long* counters, void* ws,
                          size_t ws_bytes, cudaStream_t st) {
    if (moving_cap < 1) moving_cap = 1;
    Carver cv{reinterpret_cast<char*>(ws), 0, ws_bytes};
    MergeScratch m = carve_merge(cv, moving_cap, cap, ct.tiles_total);
    if (cv.used > ws_bytes) return DASS_ERR_OOM;
    copy_len_kernel<<<1, 1, 0, st>>>(m.s.scal + 0, sb.n_moving, moving_cap);
    count_launch();
    uint32_t* keys = nullptr;
    int rc = bin_sort_core(splats, moving_cap, sb.moving, nullptr, ct, m.rec, cap, m.counters, m.s, st, &keys);
    if (rc) return rc;
    pair_depth_kernel<<<152 * 4, 256, 0, st>>>(splats, m.rec, m.counters + 2, m.depth);
    count_launch();
    tile_start_kernel<<<div_up(ct.tiles_total + 1, 256), 256, 0, st>>>(keys, m.counters + 2, ct.tiles_total, m.start);
    count_launch();
    merge_pairs_kernel<<<div_up(ct.tiles_total, kMergeWarps), 32 * kMergeWarps, 0, st>>>(
        ct.tiles_total, sb.rec, sb.depth, sb.start, sb.counters, m.rec, m.depth, m.start, m.counters, cap, pair_rec,
        tile_ranges, counters);
    count_launch();
    return check_launch("bin_sort_merge");
}

// Generic pieces reused by other translation units.
size_t scan_partials_bytes(long long len) { return sizeof(unsigned long long) * (size_t)(len / kScanTile + 2); }

int scan_u32_public(const uint32_t* in, uint32_t* out, const long long* len_dev, long long len_cap,
                    unsigned long long* partial, long long* total, cudaStream_t st) {
    return scan_u32(in, out, len_dev, len_cap, partial, total, st);
}

}  // namespace dass
