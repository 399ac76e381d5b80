// Step 5 of the binning (k_bin.cu): each tile's bucket sorted by (depth
// key, id).  Included once per block shape, with
//   BS_NS   the namespace of this instance,
//   BS_NT   threads per block (a multiple of 32, at least 256: threads
//           0..255 own the 256 digits of a pass),
//   BS_OCC  blocks per SM the kernel is compiled for.
// No include guard: the file is meant to be included more than once.

namespace BS_NS {

constexpr int BS_THREADS = BS_NT;                // threads 0..255 own digits 0..255 in the scans
constexpr int BS_WARPS = BS_THREADS / 32;
constexpr int BS_MAX = 3840;                     // bucket size sorted in shared memory
constexpr int BS_ROUNDS = BS_MAX / BS_THREADS;   // rounds of 32 per warp for a full chunk
constexpr int BS_RUN_MAX = 32;                   // longest run of equal depth keys fixed in place
// thread t owns digit t of a pass (a compile-time truth with 256 threads)
#define OWNS(t) (BS_THREADS == 256 || (t) < 256)

struct BinSortSmem {
    uint2 kv[2][BS_MAX];           // (depth key - the tile's smallest, instance id)
    uint32_t wcnt[BS_WARPS][256];  // per warp and digit: counts, then offsets within the digit
    uint32_t dbase[256];           // first position of each digit
    uint32_t run[256];             // global path: next position of each digit
    uint32_t slab[256];            // large buckets: end of each depth slab
    uint32_t sw[BS_WARPS];
    uint32_t red[4];
    uint32_t tile, flag;
};

// Digit `shift` of an entry: of its remapped depth key, or of its id - vmin.
__device__ __forceinline__ uint32_t digit_of(uint2 e, bool by_id, uint32_t vmin, int shift) {
    return ((by_id ? e.y - vmin : e.x) >> shift) & 255u;
}

// Elements per warp for a chunk of m: the chunk is split evenly, in
// multiples of 32 (a warp's round), warp w owning [w pw, (w + 1) pw).
__device__ __forceinline__ int per_warp(int m) { return ((m + BS_THREADS - 1) / BS_THREADS) * 32; }

// Stable ranking of the chunk kv[0, m) on one 8-bit digit: warp w owns
// elements [w pw, (w + 1) pw), 32 per round in order (R >= pw / 32 rounds
// unrolled); on return S.wcnt[w][d] is warp w's first position within digit
// d, and thread d holds digit d's count in `count`.
template <int R>
__device__ __forceinline__ void rank_chunk(BinSortSmem &S, const uint2 *kv, int m, bool by_id, uint32_t vmin,
                                           int shift, uint32_t (&dig)[R], uint32_t (&rank)[R], uint32_t &count) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t lt = lanemask_lt();
    for (int i = tid; i < BS_WARPS * 256; i += BS_THREADS) (&S.wcnt[0][0])[i] = 0u;
    __syncthreads();
    const int pw = per_warp(m), wb = warp * pw;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int j = wb + r * 32 + lane;
        const bool valid = r * 32 < pw && j < m;
        uint32_t d = 0;
        if (valid) d = digit_of(kv[j], by_id, vmin, shift);
        uint32_t peers = __ballot_sync(FULL, valid);
        uint32_t rk = 0;
        if (peers) {  // warp-uniform
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const uint32_t bal = __ballot_sync(FULL, (d >> b) & 1u);
                peers &= ((d >> b) & 1u) ? bal : ~bal;
            }
            uint32_t before = 0;
            if (valid) before = S.wcnt[warp][d];
            __syncwarp();
            if (valid && (peers & lt) == 0) S.wcnt[warp][d] = before + (uint32_t)__popc(peers);
            __syncwarp();
            rk = before + (uint32_t)__popc(peers & lt);
        }
        dig[r] = d;
        rank[r] = rk;
    }
    __syncthreads();
    count = 0;
    if (OWNS(tid)) {
#pragma unroll
        for (int w = 0; w < BS_WARPS; ++w) {
            const uint32_t c = S.wcnt[w][tid];
            S.wcnt[w][tid] = count;
            count += c;
        }
    }
}

// One stable pass over the chunk in shared memory: kv[src] -> kv[src ^ 1].
template <int R>
__device__ __forceinline__ void smem_pass(BinSortSmem &S, int src, int m, bool by_id, uint32_t vmin, int shift) {
    uint32_t dig[R], rank[R], count;
    rank_chunk<R>(S, S.kv[src], m, by_id, vmin, shift, dig, rank, count);
    uint32_t tot;
    const uint32_t base = block_excl_scan<BS_WARPS>(count, S.sw, tot);
    if (OWNS(threadIdx.x)) S.dbase[threadIdx.x] = base;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, pw = per_warp(m), wb = warp * pw;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int j = wb + r * 32 + lane;
        if (r * 32 < pw && j < m) S.kv[src ^ 1][S.dbase[dig[r]] + S.wcnt[warp][dig[r]] + rank[r]] = S.kv[src][j];
    }
    __syncthreads();
}

// The pass with the fewest unrolled rounds that cover m.
__device__ __forceinline__ void smem_pass_any(BinSortSmem &S, int src, int m, bool by_id, uint32_t vmin, int shift) {
    const int rounds = per_warp(m) / 32;
    if (rounds <= 1) smem_pass<1>(S, src, m, by_id, vmin, shift);
    else if (rounds <= 2) smem_pass<2>(S, src, m, by_id, vmin, shift);
    else if (rounds <= 4) smem_pass<4>(S, src, m, by_id, vmin, shift);
    else if (rounds <= 8) smem_pass<8>(S, src, m, by_id, vmin, shift);
    else if (rounds <= 12) smem_pass<12>(S, src, m, by_id, vmin, shift);
    else smem_pass<BS_ROUNDS>(S, src, m, by_id, vmin, shift);
}

// The lowest pass over the chunk, unstable: each entry's place within its
// digit comes from a returning shared-memory atomic (thread-strided entries),
// in place of the stable pass's ballot ranking and per-warp digit counts.
template <int R>
__device__ __forceinline__ void smem_pass_unstable(BinSortSmem &S, int src, int m, int shift) {
    const int tid = threadIdx.x;
    if (OWNS(tid)) S.dbase[tid] = 0u;
    __syncthreads();
    uint32_t pos[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int j = tid + r * BS_THREADS;
        pos[r] = 0u;
        if (j < m) pos[r] = atomicAdd(&S.dbase[(S.kv[src][j].x >> shift) & 255u], 1u);
    }
    __syncthreads();
    uint32_t tot;
    const uint32_t base = block_excl_scan<BS_WARPS>(OWNS(tid) ? S.dbase[tid] : 0u, S.sw, tot);
    if (OWNS(tid)) S.dbase[tid] = base;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int j = tid + r * BS_THREADS;
        if (j < m) {
            const uint2 e = S.kv[src][j];
            S.kv[src ^ 1][S.dbase[(e.x >> shift) & 255u] + pos[r]] = e;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void smem_pass_unstable_any(BinSortSmem &S, int src, int m, int shift) {
    const int rounds = (m + BS_THREADS - 1) / BS_THREADS;
    if (rounds <= 1) smem_pass_unstable<1>(S, src, m, shift);
    else if (rounds <= 2) smem_pass_unstable<2>(S, src, m, shift);
    else if (rounds <= 4) smem_pass_unstable<4>(S, src, m, shift);
    else if (rounds <= 8) smem_pass_unstable<8>(S, src, m, shift);
    else smem_pass_unstable<BS_ROUNDS>(S, src, m, shift);
}

constexpr int LD_BATCH = 8;  // global loads per thread issued together in the streaming loops

// (k - kmin, v) of entries [0, m), m <= BS_MAX, into dst: all loads of a
// thread issued before its first store, so that they are in flight together.
__device__ __forceinline__ void load_chunk(uint2 *dst, const uint32_t *k, const uint32_t *v, uint32_t m, uint32_t kmin) {
    const uint32_t tid = threadIdx.x;
    uint32_t kr[BS_ROUNDS], vr[BS_ROUNDS];
#pragma unroll
    for (int r = 0; r < BS_ROUNDS; ++r) {
        const uint32_t j = tid + r * BS_THREADS;
        kr[r] = j < m ? k[j] : 0u;
        vr[r] = j < m ? v[j] : 0u;
    }
#pragma unroll
    for (int r = 0; r < BS_ROUNDS; ++r) {
        const uint32_t j = tid + r * BS_THREADS;
        if (j < m) dst[j] = make_uint2(kr[r] - kmin, vr[r]);
    }
}

// This thread's share of the minimum and maximum of k[0, n) (and of v[0, n)
// when v is given), LD_BATCH loads in flight per step.
__device__ __forceinline__ void range_minmax(const uint32_t *k, const uint32_t *v, uint32_t n, uint32_t &kmn,
                                             uint32_t &kmx, uint32_t &vmn, uint32_t &vmx) {
    kmn = FULL; kmx = 0u; vmn = FULL; vmx = 0u;
    for (uint32_t j0 = 0; j0 < n; j0 += LD_BATCH * BS_THREADS) {
        uint32_t kr[LD_BATCH], vr[LD_BATCH];
#pragma unroll
        for (int r = 0; r < LD_BATCH; ++r) {
            const uint32_t j = j0 + threadIdx.x + r * BS_THREADS;
            kr[r] = j < n ? k[j] : FULL;
            vr[r] = (v && j < n) ? v[j] : FULL;
        }
#pragma unroll
        for (int r = 0; r < LD_BATCH; ++r) {
            const bool ok = j0 + threadIdx.x + r * BS_THREADS < n;
            if (ok) {
                kmn = min(kmn, kr[r]); kmx = max(kmx, kr[r]);
                vmn = min(vmn, vr[r]); vmx = max(vmx, vr[r]);
            }
        }
    }
    if (!v) { vmn = 0u; vmx = 0u; }
}

// One stable pass over a bucket in global memory, chunk by chunk:
// (ka, va)[0, n) -> (kb, vb)[0, n); keys are remapped by kmin while in
// shared memory.
__device__ void global_pass(BinSortSmem &S, const uint32_t *ka, const uint32_t *va, uint32_t *kb, uint32_t *vb,
                            uint32_t n, bool by_id, uint32_t kmin, uint32_t vmin, int shift) {
    const int tid = threadIdx.x;
    if (OWNS(tid)) S.dbase[tid] = 0u;
    __syncthreads();
    for (uint32_t j0 = 0; j0 < n; j0 += LD_BATCH * BS_THREADS) {  // LD_BATCH loads per thread in flight
        uint32_t d[LD_BATCH];
#pragma unroll
        for (int r = 0; r < LD_BATCH; ++r) {
            const uint32_t j = j0 + tid + r * BS_THREADS;
            d[r] = j < n ? digit_of(make_uint2(ka[j] - kmin, by_id ? va[j] : 0u), by_id, vmin, shift) : 256u;
        }
#pragma unroll
        for (int r = 0; r < LD_BATCH; ++r)
            if (d[r] < 256u) atomicAdd(&S.dbase[d[r]], 1u);
    }
    __syncthreads();
    {
        uint32_t tot;
        const uint32_t e = block_excl_scan<BS_WARPS>(OWNS(tid) ? S.dbase[tid] : 0u, S.sw, tot);
        if (OWNS(tid)) S.run[tid] = e;
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    for (uint32_t c0 = 0; c0 < n; c0 += BS_MAX) {
        const int m = (int)min((uint32_t)BS_MAX, n - c0);
        load_chunk(S.kv[0], ka + c0, va + c0, (uint32_t)m, kmin);
        __syncthreads();
        uint32_t dig[BS_ROUNDS], rank[BS_ROUNDS], count;
        rank_chunk<BS_ROUNDS>(S, S.kv[0], m, by_id, vmin, shift, dig, rank, count);
        __syncthreads();
        const int pw = per_warp(m), wb = warp * pw;
#pragma unroll
        for (int r = 0; r < BS_ROUNDS; ++r) {
            const int j = wb + r * 32 + lane;
            if (r * 32 < pw && j < m) {
                const uint32_t pos = S.run[dig[r]] + S.wcnt[warp][dig[r]] + rank[r];
                const uint2 e = S.kv[0][j];
                kb[pos] = e.x + kmin;
                vb[pos] = e.y;
            }
        }
        __syncthreads();
        if (OWNS(tid)) S.run[tid] += count;
        __syncthreads();
    }
}

// The slab split of a bucket beyond shared memory: (ka, va)[0, n) scattered
// to (kb, vb) by the digit `shift` of key - kmin, in no particular order
// within a digit (each slab is sorted afterwards, so the split need not be
// stable): the lanes of a warp with one digit reserve their places with one
// atomic.  S.run[d] ends as the end of slab d.
__device__ void global_split(BinSortSmem &S, const uint32_t *ka, const uint32_t *va, uint32_t *kb, uint32_t *vb,
                             uint32_t n, uint32_t kmin, int shift) {
    const int tid = threadIdx.x, lane = tid & 31;
    const uint32_t lt = lanemask_lt();
    if (OWNS(tid)) S.dbase[tid] = 0u;
    __syncthreads();
    for (uint32_t j0 = 0; j0 < n; j0 += LD_BATCH * BS_THREADS) {
        uint32_t d[LD_BATCH];
#pragma unroll
        for (int r = 0; r < LD_BATCH; ++r) {
            const uint32_t j = j0 + tid + r * BS_THREADS;
            d[r] = j < n ? ((ka[j] - kmin) >> shift) & 255u : 256u;
        }
#pragma unroll
        for (int r = 0; r < LD_BATCH; ++r)
            if (d[r] < 256u) atomicAdd(&S.dbase[d[r]], 1u);
    }
    __syncthreads();
    {
        uint32_t tot;
        const uint32_t e = block_excl_scan<BS_WARPS>(OWNS(tid) ? S.dbase[tid] : 0u, S.sw, tot);
        if (OWNS(tid)) S.run[tid] = e;
    }
    __syncthreads();
    for (uint32_t j0 = 0; j0 < n; j0 += LD_BATCH * BS_THREADS) {
        uint32_t kr[LD_BATCH], vr[LD_BATCH];
#pragma unroll
        for (int r = 0; r < LD_BATCH; ++r) {
            const uint32_t j = j0 + tid + r * BS_THREADS;
            kr[r] = j < n ? ka[j] : 0u;
            vr[r] = j < n ? va[j] : 0u;
        }
#pragma unroll
        for (int r = 0; r < LD_BATCH; ++r) {
            const bool valid = j0 + tid + r * BS_THREADS < n;
            uint32_t peers = __ballot_sync(FULL, valid);
            if (peers) {  // warp-uniform
                const uint32_t d = ((kr[r] - kmin) >> shift) & 255u;
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    const uint32_t bal = __ballot_sync(FULL, (d >> b) & 1u);
                    peers &= ((d >> b) & 1u) ? bal : ~bal;
                }
                const int leader = peers ? __ffs(peers) - 1 : lane;
                uint32_t base = 0;
                if (valid && lane == leader) base = atomicAdd(&S.run[d], (uint32_t)__popc(peers));
                base = __shfl_sync(FULL, base, leader);
                if (valid) {
                    const uint32_t pos = base + (uint32_t)__popc(peers & lt);
                    kb[pos] = kr[r];
                    vb[pos] = vr[r];
                }
            }
        }
    }
    __syncthreads();
}

__device__ __forceinline__ int sig_bits(uint32_t lo, uint32_t hi) { return hi > lo ? 32 - __clz(hi - lo) : 0; }

// Block-wide min and max of two words (results in S.red: kmin, kmax, vmin, vmax).
__device__ __forceinline__ void block_minmax(BinSortSmem &S, uint32_t kmn, uint32_t kmx, uint32_t vmn, uint32_t vmx) {
    kmn = __reduce_min_sync(FULL, kmn);
    kmx = __reduce_max_sync(FULL, kmx);
    vmn = __reduce_min_sync(FULL, vmn);
    vmx = __reduce_max_sync(FULL, vmx);
    if (threadIdx.x == 0) {
        S.red[0] = FULL;
        S.red[1] = 0u;
        S.red[2] = FULL;
        S.red[3] = 0u;
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&S.red[0], kmn);
        atomicMax(&S.red[1], kmx);
        atomicMin(&S.red[2], vmn);
        atomicMax(&S.red[3], vmx);
    }
    __syncthreads();
}

// Entries in global memory (two arrays).
struct GlobalEntries {
    const uint32_t *k;
    uint32_t *v;
    __device__ uint32_t key(uint32_t j) const { return k[j]; }
    __device__ uint32_t id(uint32_t j) const { return v[j]; }
    __device__ void set_id(uint32_t j, uint32_t x) const { v[j] = x; }
};

// Puts the ids of each run of equal keys of entries [0, n) (sorted by key)
// in ascending order, in place, when the run holds at most 32 entries (one
// thread per run); returns true (block-uniform) when a longer run exists,
// leaving the entries sorted by key only.
template <class E>
__device__ bool fix_ties(BinSortSmem &S, const E &e, uint32_t n) {
    const int tid = threadIdx.x;
    if (tid == 0) S.flag = 0u;
    __syncthreads();
    for (uint32_t j = tid; j + 1 < n; j += BS_THREADS) {
        const uint32_t kj = e.key(j);
        if ((j == 0 || e.key(j - 1) != kj) && e.key(j + 1) == kj) {
            uint32_t end = j + 1;
            while (end < n && e.key(end) == kj && end - j <= (uint32_t)BS_RUN_MAX) ++end;
            if (end - j > (uint32_t)BS_RUN_MAX) {
                atomicOr(&S.flag, 1u);
            } else {
                for (uint32_t x = j + 1; x < end; ++x) {  // insertion sort of the run's ids
                    const uint32_t vx = e.id(x);
                    uint32_t y = x;
                    while (y > j && e.id(y - 1) > vx) {
                        e.set_id(y, e.id(y - 1));
                        --y;
                    }
                    e.set_id(y, vx);
                }
            }
        }
    }
    __syncthreads();
    const bool longrun = S.flag != 0u;
    __syncthreads();
    return longrun;
}

// Puts each run of entries with equal key >> lo (entries [0, n) in shared
// memory, sorted by key >> lo) in (key, id) order, in place, when the run
// holds at most BS_RUN_MAX entries (one thread per run, insertion); returns
// true (block-uniform) when a longer run exists, leaving it as it was.
__device__ bool fix_runs(BinSortSmem &S, uint2 *kv, uint32_t n, int lo) {
    const int tid = threadIdx.x;
    if (tid == 0) S.flag = 0u;
    __syncthreads();
    for (uint32_t j = tid; j + 1 < n; j += BS_THREADS) {
        const uint32_t hj = kv[j].x >> lo;
        if ((j == 0 || (kv[j - 1].x >> lo) != hj) && (kv[j + 1].x >> lo) == hj) {
            uint32_t end = j + 1;
            while (end < n && (kv[end].x >> lo) == hj && end - j <= (uint32_t)BS_RUN_MAX) ++end;
            if (end - j > (uint32_t)BS_RUN_MAX) {
                atomicOr(&S.flag, 1u);
            } else {
                for (uint32_t x = j + 1; x < end; ++x) {
                    const uint2 vx = kv[x];
                    uint32_t y = x;
                    while (y > j && (kv[y - 1].x > vx.x || (kv[y - 1].x == vx.x && kv[y - 1].y > vx.y))) {
                        kv[y] = kv[y - 1];
                        --y;
                    }
                    kv[y] = vx;
                }
            }
        }
    }
    __syncthreads();
    const bool longrun = S.flag != 0u;
    __syncthreads();
    return longrun;
}

// Sorts n <= BS_MAX entries (keys k, ids v in global memory) by (key, id)
// in shared memory and writes the ids to out (which may alias v).  The radix
// passes cover the highest 8 * npass significant key bits (npass = 2 up to
// 24 significant bits, else 3); runs of entries that agree on those bits are
// then put in (key, id) order by insertion, which completes the order.  The
// lowest pass need not be stable: the order it leaves among entries of one
// digit survives the stable passes above it only within such runs, which
// the insertion re-sorts.
__device__ void sort_range_smem(BinSortSmem &S, const uint32_t *k, const uint32_t *v, uint32_t n, uint32_t *out) {
    const int tid = threadIdx.x;
    if (n <= 1) {
        if (n == 1 && tid == 0) out[0] = v[0];
        __syncthreads();
        return;
    }
    // the whole bucket in registers first (BS_ROUNDS loads per thread in flight together)
    uint32_t kr[BS_ROUNDS], vr[BS_ROUNDS];
#pragma unroll
    for (int r = 0; r < BS_ROUNDS; ++r) {
        const uint32_t j = tid + r * BS_THREADS;
        kr[r] = j < n ? k[j] : 0u;
        vr[r] = j < n ? v[j] : 0u;
    }
    uint32_t kmn = FULL, kmx = 0u, vmn = FULL, vmx = 0u;
#pragma unroll
    for (int r = 0; r < BS_ROUNDS; ++r)
        if (tid + r * BS_THREADS < n) {
            kmn = min(kmn, kr[r]); kmx = max(kmx, kr[r]); vmn = min(vmn, vr[r]); vmx = max(vmx, vr[r]);
        }
    block_minmax(S, kmn, kmx, vmn, vmx);
    const uint32_t kmin = S.red[0], vmin = S.red[2];
    const int kb = sig_bits(kmin, S.red[1]), vb = sig_bits(vmin, S.red[3]);
    const int m = (int)n;
#pragma unroll
    for (int r = 0; r < BS_ROUNDS; ++r) {
        const uint32_t j = tid + r * BS_THREADS;
        if (j < n) S.kv[0][j] = make_uint2(kr[r] - kmin, vr[r]);
    }
    __syncthreads();
    int src = 0;
    const int npass = kb <= 16 ? (kb + 7) / 8 : (kb <= 24 ? 2 : 3);
    const int lo = max(0, kb - 8 * npass);  // key bits below the passes
    for (int sh = lo; sh < kb; sh += 8) {
        if (sh == lo) smem_pass_unstable_any(S, src, m, sh);
        else smem_pass_any(S, src, m, false, vmin, sh);
        src ^= 1;
    }
    // runs that agree on the passes' bits: (key, id) order (short runs in place)
    if (fix_runs(S, S.kv[src], n, lo)) {  // a long run: the full (depth key, id) order
        for (int sh = 0; sh < vb; sh += 8) {
            smem_pass_any(S, src, m, true, vmin, sh);
            src ^= 1;
        }
        for (int sh = 0; sh < kb; sh += 8) {
            smem_pass_any(S, src, m, false, vmin, sh);
            src ^= 1;
        }
    }
    for (int j = tid; j < m; j += BS_THREADS) out[j] = S.kv[src][j].y;
    __syncthreads();
}

// Sorts n entries by radix passes over global memory: (k0, v0) with the
// scratch (k1, v1); ids to out (which may alias v0 or v1).
__device__ void sort_range_global(BinSortSmem &S, uint32_t *k0, uint32_t *v0, uint32_t *k1, uint32_t *v1, uint32_t n,
                                  uint32_t *out) {
    const int tid = threadIdx.x;
    uint32_t kmn, kmx, vmn, vmx;
    range_minmax(k0, v0, n, kmn, kmx, vmn, vmx);
    block_minmax(S, kmn, kmx, vmn, vmx);
    const uint32_t kmin = S.red[0], vmin = S.red[2];
    const int kb = sig_bits(kmin, S.red[1]), vb = sig_bits(vmin, S.red[3]);
    for (int sh = 0; sh < kb; sh += 8) {
        global_pass(S, k0, v0, k1, v1, n, false, kmin, vmin, sh);
        uint32_t *t = k0; k0 = k1; k1 = t;
        t = v0; v0 = v1; v1 = t;
    }
    if (fix_ties(S, GlobalEntries{k0, v0}, n)) {  // a long run of equal depth keys: ids, then depth
        for (int sh = 0; sh < vb; sh += 8) {
            global_pass(S, k0, v0, k1, v1, n, true, kmin, vmin, sh);
            uint32_t *t = k0; k0 = k1; k1 = t;
            t = v0; v0 = v1; v1 = t;
        }
        for (int sh = 0; sh < kb; sh += 8) {
            global_pass(S, k0, v0, k1, v1, n, false, kmin, vmin, sh);
            uint32_t *t = k0; k0 = k1; k1 = t;
            t = v0; v0 = v1; v1 = t;
        }
    }
    if (out != v0) {  // the result is in (k0, v0)
        for (uint32_t j0 = 0; j0 < n; j0 += LD_BATCH * BS_THREADS) {
            uint32_t vr[LD_BATCH];
#pragma unroll
            for (int r = 0; r < LD_BATCH; ++r) {
                const uint32_t j = j0 + tid + r * BS_THREADS;
                vr[r] = j < n ? v0[j] : 0u;
            }
#pragma unroll
            for (int r = 0; r < LD_BATCH; ++r) {
                const uint32_t j = j0 + tid + r * BS_THREADS;
                if (j < n) out[j] = vr[r];
            }
        }
    }
    __syncthreads();
}

__global__ __launch_bounds__(BS_THREADS, BS_OCC) void k_bin_sort(BinArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BinSortSmem &S = *reinterpret_cast<BinSortSmem *>(smem_raw);
    const int tid = threadIdx.x;
    if (*a.p_dev > a.p_cap) return;  // nothing was filled (the ranges are empty)
    for (;;) {
        if (tid == 0) S.tile = atomicAdd(a.tile_ctr, 1u);
        __syncthreads();
        const uint32_t q = S.tile;
        __syncthreads();
        if (q >= a.n_slots) break;
        const uint2 rg = a.ranges[a.tile_order[q]];
        const uint32_t first = rg.x, n = rg.y - rg.x;
        if (n == 0) continue;
        uint32_t *bk = a.bk_key + first, *bi = a.bk_id + first;
        uint32_t *tk = a.tmp_key + first, *ti = a.tmp_id + first;
        uint32_t *out = a.ids_out + first;
        if (n <= (uint32_t)BS_MAX) {
            sort_range_smem(S, bk, bi, n, out);
            continue;
        }
        // A bucket beyond shared memory: one unstable pass over global memory
        // on the highest significant digit splits it into depth slabs; runs of
        // consecutive slabs of at most BS_MAX entries are then sorted in
        // shared memory, and a slab larger than that by global passes.
        uint32_t kmn, kmx, vmn, vmx;
        range_minmax(bk, nullptr, n, kmn, kmx, vmn, vmx);
        block_minmax(S, kmn, kmx, vmn, vmx);
        const uint32_t kmin = S.red[0];
        const int kb = sig_bits(kmin, S.red[1]);
        if (kb == 0) {  // one depth key: the id order, by global passes
            sort_range_global(S, bk, bi, tk, ti, n, out);
            continue;
        }
        global_split(S, bk, bi, tk, ti, n, kmin, ((kb - 1) / 8) * 8);
        if (OWNS(tid)) S.slab[tid] = S.run[tid];  // end of each slab (the passes below reuse S.run)
        __syncthreads();
        uint32_t c0 = 0;  // start of the pending run of slabs (the same in every thread)
        for (int d = 0; d < 256; ++d) {
            const uint32_t beg = d ? S.slab[d - 1] : 0u, end = S.slab[d];
            if (end - c0 <= (uint32_t)BS_MAX) continue;
            if (beg > c0) sort_range_smem(S, tk + c0, ti + c0, beg - c0, out + c0);
            c0 = beg;
            if (end - beg > (uint32_t)BS_MAX) {
                sort_range_global(S, tk + beg, ti + beg, bk + beg, bi + beg, end - beg, out + beg);
                c0 = end;
            }
        }
        if (n > c0) sort_range_smem(S, tk + c0, ti + c0, n - c0, out + c0);
    }
}


// Kernel attributes (once per device) and the grid: every SM the kernel's
// occupancy allows.
int setup() {
    static PerDevice cache;
    return cache.get([](int) {
        const size_t smem = sizeof(BinSortSmem);
        cudaFuncSetAttribute(k_bin_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bin_sort, BS_THREADS, smem);
        return sm_count() * std::max(1, per_sm);
    });
}

void launch(const BinArgs &a, cudaStream_t s) {
    const int grid = setup();
    cudaMemsetAsync(a.tile_ctr, 0, sizeof(uint32_t), s);
    k_bin_sort<<<std::min(grid, (int)std::max<uint32_t>(a.n_slots, 1)), BS_THREADS, sizeof(BinSortSmem), s>>>(a);
}

}  // namespace BS_NS

#undef OWNS
