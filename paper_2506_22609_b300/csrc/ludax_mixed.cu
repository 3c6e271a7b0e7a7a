// ludax_mixed.cu -- mixed-game batches in one persistent launch, the CUDA
// graph plan that replays it, and the launch-shape autotuner.
//
// Each env carries an int32 descriptor game | rows << 8 | cols << 16 (plus
// line << 24 | flags << 28 for the line game).  At plan creation the env ids
// are grouped by kernel instance ("buckets": Tic-Tac-Toe, Connect Four,
// Reversi, Hex 2..11, Gomoku, Pente, Yavalath, the parametric line game, Wolf
// and Sheep, Draughts, Dai Hasami Shogi) into a work queue, so consecutive
// queue positions -- and therefore the 32 lanes of a warp -- play the same
// game and branch together.  With a thread per env the hardware's block
// scheduler hands out the work; a persistent launch (fewer threads than
// envs) gives each bucket its own warp-aggregated atomic cursor: a warp
// stays inside one bucket, a lane whose game ends writes its 3 bytes of
// output and claims that bucket's next position, and once the bucket is
// drained the warp moves on to the next bucket with work.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>
#include <vector>

#include "ludax_internal.cuh"

using namespace ludax;

namespace {

constexpr int kBuckets = kDescBuckets;
// Buckets in decreasing order of the time one env takes to play out (single-
// game launches of 65,536 envs: Dai Hasami Shogi, Pente, Draughts, Gomoku,
// Hex 11, the line game, Reversi, Hex 10, Hex 9, Wolf and Sheep, ...,
// Tic-Tac-Toe, Hex 3, Hex 2).  The one-env-per-thread launch starts the
// buckets in this order (six-game mix 0.851 -> 0.812 ms, the 13 library
// games 4.61 ms persistent -> 3.97 ms).
__device__ constexpr int kLongestFirst[kBuckets] = {19, 14, 18, 13, 12, 16, 2, 11, 10, 17,
                                                    9, 8, 15, 7, 1, 6, 5, 0, 4, 3};
constexpr int kHexTableCells = 505;  // sum of n*n for n = 2..11

__host__ __device__ constexpr int hex_table_offset(int n) {
    int off = 0;
    for (int k = 2; k < n; ++k) off += k * k;
    return off;
}

int bucket_of_desc(int32_t d) { return desc_bucket(d); }

struct MixedArgs {
    const int32_t* queue;            // env ids grouped by bucket
    const int32_t* desc;             // per-env descriptors (parameters of the line game)
    long long bucket_end[kBuckets];  // exclusive end position of each bucket in the queue
    long long n;
    long long env_offset;
    uint64_t seed_key;
    int8_t* outcome;
    int16_t* plies;
    unsigned long long* cursor;      // per-bucket claim cursors, zeroed before each launch
    const long long* bucket_end_dev; // non-null: the bucket ends were built on the device (host-buffer path)
    int lanes;                       // one-thread-per-env launch: lanes of each warp that hold envs (8, 16, 32)
};
// The mixed kernel takes exactly one parameter (MixedArgs): the graph plan
// rewrites that single parameter before each replay.

// Every block first copies the bucket ends into shared memory (from the
// kernel parameter, or from device memory when the queue was built on the
// device), and the helpers below read them there.
__device__ __forceinline__ void load_bucket_ends(const MixedArgs& a, long long* be) {
    if (threadIdx.x < kBuckets) be[threadIdx.x] = a.bucket_end_dev ? a.bucket_end_dev[threadIdx.x] : a.bucket_end[threadIdx.x];
}

__device__ __forceinline__ int bucket_at(const long long* be, long long q) {
    int b = 0;
#pragma unroll
    for (int k = 0; k < kBuckets - 1; ++k) b += q >= be[k];
    return b;
}

// Non-persistent launches (a thread per env, the hardware's block scheduler
// refilling the SMs): plays the env at queue position q to its end.
template <class G>
__device__ __forceinline__ void play_one(const MixedArgs& a, long long q, const B128* table) {
    G g;
    set_table(g, table);
    const long long e = a.queue[q];
    configure(g, a.desc[e]);
    g.reset();
    const uint64_t key = env_key(a.seed_key, (uint64_t)(a.env_offset + e));
    uint32_t rhi = draw_hi(key, 0u);
    while (g.outcome == kOngoing) random_ply_pre(g, key, rhi);
    a.outcome[e] = (int8_t)g.outcome;
    a.plies[e] = (int16_t)g.ply;
}

// The same for two envs of one bucket per thread (queue positions q0 and
// q1, q1 < 0 for none), interleaved ply by ply: two independent dependency
// chains in each thread (the "unroll").
template <class G>
__device__ __forceinline__ void play_pair(const MixedArgs& a, long long q0, long long q1, const B128* table) {
    G g[2];
    uint64_t key[2];
    uint32_t rhi[2];
    long long e[2];
    bool on[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const long long q = i ? q1 : q0;
        set_table(g[i], table);
        on[i] = q >= 0;
        e[i] = on[i] ? a.queue[q] : 0;
        if (on[i]) configure(g[i], a.desc[e[i]]);
        g[i].reset();
        key[i] = env_key(a.seed_key, (uint64_t)(a.env_offset + e[i]));
        rhi[i] = draw_hi(key[i], 0u);
    }
    for (;;) {
        bool any = false;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            if (!on[i]) continue;
            any = true;
            if (g[i].outcome == kOngoing) {
                random_ply_pre(g[i], key[i], rhi[i]);
                continue;
            }
            a.outcome[e[i]] = (int8_t)g[i].outcome;
            a.plies[e[i]] = (int16_t)g[i].ply;
            on[i] = false;
        }
        if (!any) break;
    }
}

template <class G, int EPT>
__device__ __forceinline__ void play_n(const MixedArgs& a, long long q0, long long q1, const B128* table) {
    if constexpr (EPT == 1) play_one<G>(a, q0, table);
    else play_pair<G>(a, q0, q1, table);
}

// the game of bucket b, for the positions q0 (and q1 with EPT 2)
template <bool TABLE, int EPT>
__device__ __forceinline__ void play_bucket(const MixedArgs& a, int b, long long q0, long long q1, const B128* t) {
    switch (b) {
    case 0: play_n<TTT, EPT>(a, q0, q1, nullptr); break;
    case 1: play_n<C4, EPT>(a, q0, q1, nullptr); break;
    case 2: play_n<Othello, EPT>(a, q0, q1, nullptr); break;
    case 3: play_n<Hex<2>, EPT>(a, q0, q1, TABLE ? t + hex_table_offset(2) : nullptr); break;
    case 4: play_n<Hex<3>, EPT>(a, q0, q1, TABLE ? t + hex_table_offset(3) : nullptr); break;
    case 5: play_n<Hex<4>, EPT>(a, q0, q1, TABLE ? t + hex_table_offset(4) : nullptr); break;
    case 6: play_n<Hex<5>, EPT>(a, q0, q1, TABLE ? t + hex_table_offset(5) : nullptr); break;
    case 7: play_n<Hex<6>, EPT>(a, q0, q1, TABLE ? t + hex_table_offset(6) : nullptr); break;
    case 8: play_n<Hex<7>, EPT>(a, q0, q1, TABLE ? t + hex_table_offset(7) : nullptr); break;
    case 9: play_n<Hex<8>, EPT>(a, q0, q1, TABLE ? t + hex_table_offset(8) : nullptr); break;
    case 10: play_n<Hex<9>, EPT>(a, q0, q1, TABLE ? t + hex_table_offset(9) : nullptr); break;
    case 11: play_n<Hex<10>, EPT>(a, q0, q1, TABLE ? t + hex_table_offset(10) : nullptr); break;
    case 12: play_n<Hex<11>, EPT>(a, q0, q1, TABLE ? t + hex_table_offset(11) : nullptr); break;
    case 13: play_n<Gomoku, EPT>(a, q0, q1, nullptr); break;
    case 14: play_n<Pente, EPT>(a, q0, q1, nullptr); break;
    case 15: play_n<Yavalath, EPT>(a, q0, q1, nullptr); break;
    case 16: play_n<LineGame, EPT>(a, q0, q1, nullptr); break;
    case 17: play_n<WolfSheep, EPT>(a, q0, q1, nullptr); break;
    case 18: play_n<Draughts, EPT>(a, q0, q1, nullptr); break;
    default: play_n<HasamiShogi, EPT>(a, q0, q1, nullptr); break;
    }
}

// Persistent launches: a warp stays inside one bucket (one game, so its
// lanes branch together) and its lanes take that bucket's positions from the
// bucket's own cursor, one new env per finished lane, until the bucket is
// drained; then the warp moves on to the next bucket with work.  (A single
// cursor over the whole queue would let the lanes of a warp drift into
// different games.)
__device__ __forceinline__ long long bucket_begin(const long long* be, int b) { return b == 0 ? 0 : be[b - 1]; }

// positions for the lanes in `want` from bucket b's cursor (warp-aggregated);
// a result >= the bucket's end means the bucket is drained
__device__ __forceinline__ long long claim_in_bucket(const MixedArgs& a, const long long* be, int b, bool want) {
    const unsigned m = __ballot_sync(0xFFFFFFFFu, want);
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (m && lane == leader) base = atomicAdd(&a.cursor[b], (unsigned long long)__popc(m));
    base = __shfl_sync(0xFFFFFFFFu, base, leader < 0 ? 0 : leader);
    return bucket_begin(be, b) + (long long)(base + __popc(m & ((1u << lane) - 1u)));
}

// One lane plays positions of bucket b, from its first claim q, taking the
// next position from the bucket's cursor when a game ends (the lanes that
// finish together claim with one atomic), until the bucket is drained.
template <class G>
__device__ __forceinline__ void drain_bucket(const MixedArgs& a, const long long* be, int b, long long q,
                                             const B128* table) {
    const long long begin = bucket_begin(be, b), end = be[b];
    G g;
    set_table(g, table);
    long long e = a.queue[q];
    configure(g, a.desc[e]);
    g.reset();
    uint64_t key = env_key(a.seed_key, (uint64_t)(a.env_offset + e));
    uint32_t rhi = draw_hi(key, 0u);
    for (;;) {
        if (g.outcome == kOngoing) {
            random_ply_pre(g, key, rhi);
            continue;
        }
        a.outcome[e] = (int8_t)g.outcome;
        a.plies[e] = (int16_t)g.ply;
        q = begin + claim_next(&a.cursor[b]);
        if (q >= end) return;
        e = a.queue[q];
        configure(g, a.desc[e]);
        g.reset();
        key = env_key(a.seed_key, (uint64_t)(a.env_offset + e));
        rhi = draw_hi(key, 0u);
    }
}

template <bool TABLE>
__device__ __forceinline__ void drain_any(const MixedArgs& a, const long long* be, int b, long long q,
                                          const B128* tables) {
    switch (b) {
    case 0: drain_bucket<TTT>(a, be, b, q, nullptr); break;
    case 1: drain_bucket<C4>(a, be, b, q, nullptr); break;
    case 2: drain_bucket<Othello>(a, be, b, q, nullptr); break;
    case 3: drain_bucket<Hex<2>>(a, be, b, q, TABLE ? tables + hex_table_offset(2) : nullptr); break;
    case 4: drain_bucket<Hex<3>>(a, be, b, q, TABLE ? tables + hex_table_offset(3) : nullptr); break;
    case 5: drain_bucket<Hex<4>>(a, be, b, q, TABLE ? tables + hex_table_offset(4) : nullptr); break;
    case 6: drain_bucket<Hex<5>>(a, be, b, q, TABLE ? tables + hex_table_offset(5) : nullptr); break;
    case 7: drain_bucket<Hex<6>>(a, be, b, q, TABLE ? tables + hex_table_offset(6) : nullptr); break;
    case 8: drain_bucket<Hex<7>>(a, be, b, q, TABLE ? tables + hex_table_offset(7) : nullptr); break;
    case 9: drain_bucket<Hex<8>>(a, be, b, q, TABLE ? tables + hex_table_offset(8) : nullptr); break;
    case 10: drain_bucket<Hex<9>>(a, be, b, q, TABLE ? tables + hex_table_offset(9) : nullptr); break;
    case 11: drain_bucket<Hex<10>>(a, be, b, q, TABLE ? tables + hex_table_offset(10) : nullptr); break;
    case 12: drain_bucket<Hex<11>>(a, be, b, q, TABLE ? tables + hex_table_offset(11) : nullptr); break;
    case 13: drain_bucket<Gomoku>(a, be, b, q, nullptr); break;
    case 14: drain_bucket<Pente>(a, be, b, q, nullptr); break;
    case 15: drain_bucket<Yavalath>(a, be, b, q, nullptr); break;
    case 16: drain_bucket<LineGame>(a, be, b, q, nullptr); break;
    case 17: drain_bucket<WolfSheep>(a, be, b, q, nullptr); break;
    case 18: drain_bucket<Draughts>(a, be, b, q, nullptr); break;
    default: drain_bucket<HasamiShogi>(a, be, b, q, nullptr); break;
    }
}

// One thread per env (EPT envs per thread, interleaved); only the first
// a.lanes lanes of each warp hold envs.  A block covers EPT runs of
// (blockDim / 32) * a.lanes consecutive positions; a thread takes its slot in
// each run, so its envs are nearly always of one bucket (when they are not,
// it plays them one after the other).
template <bool TABLE, int EPT>
__global__ void __launch_bounds__(512) mixed_rollout_kernel(MixedArgs a) {
    __shared__ B128 tables[TABLE ? kHexTableCells : 1];
    if constexpr (TABLE) {
        hex_fill_table<2>(tables + hex_table_offset(2));
        hex_fill_table<3>(tables + hex_table_offset(3));
        hex_fill_table<4>(tables + hex_table_offset(4));
        hex_fill_table<5>(tables + hex_table_offset(5));
        hex_fill_table<6>(tables + hex_table_offset(6));
        hex_fill_table<7>(tables + hex_table_offset(7));
        hex_fill_table<8>(tables + hex_table_offset(8));
        hex_fill_table<9>(tables + hex_table_offset(9));
        hex_fill_table<10>(tables + hex_table_offset(10));
        hex_fill_table<11>(tables + hex_table_offset(11));
        __syncthreads();
    }
    __shared__ long long be[kBuckets], seg_end[kBuckets], seg_q[kBuckets];
    load_bucket_ends(a, be);
    __syncthreads();
    // Blocks are handed out in index order, so thread position q0 walks the
    // buckets in kLongestFirst order: the games that take longest start first
    // and the short ones fill the tail of the launch (longest-first
    // scheduling).  seg_end[i] = positions covered by the first i + 1 buckets
    // of that order, seg_q[i] = queue offset of segment i.
    if (threadIdx.x == 0) {
        long long acc = 0;
        for (int i = 0; i < kBuckets; ++i) {
            const int b = kLongestFirst[i];
            const long long beg = b == 0 ? 0 : be[b - 1];
            seg_q[i] = beg - acc;
            acc += be[b] - beg;
            seg_end[i] = acc;
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    if (lane >= a.lanes) return;
    const long long run = (long long)(blockDim.x >> 5) * a.lanes;
    const long long slot = (long long)(threadIdx.x >> 5) * a.lanes + lane;
    long long q[EPT];
    int b[EPT];
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
        const long long q0 = (long long)blockIdx.x * run * EPT + i * run + slot;
        q[i] = -1;
        b[i] = -1;
        if (q0 >= be[kBuckets - 1]) continue;  // past the last valid queue position
        int si = 0;
#pragma unroll
        for (int k = 0; k < kBuckets - 1; ++k) si += q0 >= seg_end[k];
        q[i] = q0 + seg_q[si];
        b[i] = bucket_at(be, q[i]);
    }
    if (q[0] < 0) return;
    if constexpr (EPT == 1) {
        play_bucket<TABLE, 1>(a, b[0], q[0], -1, tables);
    } else if (q[1] < 0 || b[1] == b[0]) {
        play_bucket<TABLE, 2>(a, b[0], q[0], q[1], tables);
    } else {  // a bucket boundary between the two: one after the other
        play_bucket<TABLE, 2>(a, b[0], q[0], -1, tables);
        play_bucket<TABLE, 2>(a, b[1], q[1], -1, tables);
    }
}

// Persistent launches (fewer threads than envs): warps drain buckets,
// starting spread over the queue in proportion to the buckets' sizes.
template <bool TABLE>
__global__ void __launch_bounds__(512, 1) mixed_persistent_kernel(MixedArgs a) {
    __shared__ B128 tables[TABLE ? kHexTableCells : 1];
    if constexpr (TABLE) {
        hex_fill_table<2>(tables + hex_table_offset(2));
        hex_fill_table<3>(tables + hex_table_offset(3));
        hex_fill_table<4>(tables + hex_table_offset(4));
        hex_fill_table<5>(tables + hex_table_offset(5));
        hex_fill_table<6>(tables + hex_table_offset(6));
        hex_fill_table<7>(tables + hex_table_offset(7));
        hex_fill_table<8>(tables + hex_table_offset(8));
        hex_fill_table<9>(tables + hex_table_offset(9));
        hex_fill_table<10>(tables + hex_table_offset(10));
        hex_fill_table<11>(tables + hex_table_offset(11));
        __syncthreads();
    }
    __shared__ long long be[kBuckets];
    load_bucket_ends(a, be);
    __syncthreads();
    const long long slots = (long long)gridDim.x * blockDim.x;
    const long long warps = slots >> 5, w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int b = bucket_at(be, w * be[kBuckets - 1] / warps);
    for (int idle = 0; idle < kBuckets; b = (b + 1) % kBuckets) {
        const long long q = claim_in_bucket(a, be, b, true);  // the whole warp enters bucket b together
        const bool mine = q < be[b];
        if (__any_sync(0xFFFFFFFFu, mine)) {
            idle = 0;
            if (mine) drain_any<TABLE>(a, be, b, q, tables);
        } else {
            ++idle;
        }
        __syncwarp();  // lanes leave the bucket together
    }
}

int mixed_lanes(const ludax_launch_cfg& c) {
    return (c.lanes_per_warp == 8 || c.lanes_per_warp == 16) ? c.lanes_per_warp : 32;
}

int mixed_grid(long long n, const ludax_launch_cfg& c, int num_sms) {
    const long long per_block = (long long)(c.block_threads / 32) * mixed_lanes(c) * c.envs_per_thread;
    long long need = (n + per_block - 1) / per_block;
    if (c.blocks_per_sm > 0) need = std::min<long long>(need, (long long)num_sms * c.blocks_per_sm);
    return (int)std::max<long long>(need, 1);
}

int check_mixed_cfg(const ludax_launch_cfg& c) {
    if (c.block_threads < 32 || c.block_threads > 512 || c.block_threads % 32) return LUDAX_ERR_ARG;
    if (c.blocks_per_sm < 0 || c.blocks_per_sm > 64) return LUDAX_ERR_ARG;
    if (c.envs_per_thread != 1 && c.envs_per_thread != 2) return LUDAX_ERR_ARG;
    if (c.lanes_per_warp != 0 && c.lanes_per_warp != 8 && c.lanes_per_warp != 16 && c.lanes_per_warp != 32)
        return LUDAX_ERR_ARG;
    // two envs per thread and part-filled warps: one-thread-per-env launches only
    if ((c.envs_per_thread != 1 || mixed_lanes(c) != 32) && c.blocks_per_sm != 0) return LUDAX_ERR_ARG;
    if (c.hex_nbr_table != 0 && c.hex_nbr_table != 1) return LUDAX_ERR_ARG;
    if (c.compact_every != 0) return LUDAX_ERR_ARG;  // compaction is a single-game option
    if (c.threads_per_env > 1 || c.threads_per_env < 0) return LUDAX_ERR_ARG;  // one lane per env
    return LUDAX_OK;
}

// Groups env ids by bucket on the host (stable: ascending env id inside a
// bucket).  Returns LUDAX_OK or the error of the first bad descriptor.
int build_queue(const int32_t* desc_dev, long long n, std::vector<int32_t>& queue, long long* bucket_end,
                int64_t* bad_index) {
    std::vector<int32_t> desc((size_t)n);
    if (cudaMemcpy(desc.data(), desc_dev, sizeof(int32_t) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
        return LUDAX_ERR_CUDA;
    long long count[kBuckets] = {0};
    for (long long e = 0; e < n; ++e) {
        int b = bucket_of_desc(desc[(size_t)e]);
        if (b < 0) {
            if (bad_index) *bad_index = e;
            return b == -1 ? LUDAX_ERR_GAME : LUDAX_ERR_SIZE;
        }
        count[b]++;
    }
    long long pos[kBuckets], acc = 0;
    for (int b = 0; b < kBuckets; ++b) {
        pos[b] = acc;
        acc += count[b];
        bucket_end[b] = acc;
    }
    queue.resize((size_t)n);
    for (long long e = 0; e < n; ++e) queue[(size_t)pos[bucket_of_desc(desc[(size_t)e])]++] = (int32_t)e;
    if (bad_index) *bad_index = -1;
    return LUDAX_OK;
}

int launch_mixed(MixedArgs a, const ludax_launch_cfg& c, int num_sms, cudaStream_t s) {
    int grid = mixed_grid(a.n, c, num_sms);
    a.lanes = mixed_lanes(c);
    if (cudaMemsetAsync(a.cursor, 0, sizeof(unsigned long long) * kBuckets, s) != cudaSuccess) return LUDAX_ERR_CUDA;
    if ((long long)grid * c.block_threads < a.n) {  // persistent (full warps, one env per thread)
        if (c.hex_nbr_table) mixed_persistent_kernel<true><<<grid, c.block_threads, 0, s>>>(a);
        else mixed_persistent_kernel<false><<<grid, c.block_threads, 0, s>>>(a);
    } else if (c.envs_per_thread == 2) {
        if (c.hex_nbr_table) mixed_rollout_kernel<true, 2><<<grid, c.block_threads, 0, s>>>(a);
        else mixed_rollout_kernel<false, 2><<<grid, c.block_threads, 0, s>>>(a);
    } else if (c.hex_nbr_table) {
        mixed_rollout_kernel<true, 1><<<grid, c.block_threads, 0, s>>>(a);
    } else {
        mixed_rollout_kernel<false, 1><<<grid, c.block_threads, 0, s>>>(a);
    }
    return cudaGetLastError() == cudaSuccess ? LUDAX_OK : LUDAX_ERR_CUDA;
}

int num_sms_current(int* out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LUDAX_ERR_CUDA;
    if (cudaDeviceGetAttribute(out, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LUDAX_ERR_CUDA;
    return LUDAX_OK;
}

ludax_launch_cfg default_mixed_cfg() { return ludax_launch_cfg{256, 0, 1, 0, 0}; }

}  // namespace

// Host-buffer launches (ludax_mixed_plan_launch_host) build the work queue on
// the device from the uploaded descriptors: a histogram of the buckets (and
// the first invalid descriptor), one block turning it into bucket ends, and a
// scatter of the env ids; the playout kernel then reads the bucket ends from
// device memory.  Counter words: [0, 20) claim cursors, [20, 40) bucket
// counts, [40, 60) fill positions, [60] first invalid index (all ones: none).
namespace {
constexpr int kHostCtrWords = 64, kHostCount = 20, kHostFill = 40, kHostBad = 60;
static_assert(kBuckets <= 20, "counter layout holds 20 buckets");

__global__ void hq_init_kernel(unsigned long long* ctr) {
    if (threadIdx.x < kHostCtrWords) ctr[threadIdx.x] = threadIdx.x == kHostBad ? ~0ull : 0ull;
}

// bucket histogram (block-local, one atomic per bucket per block); an env
// with an invalid descriptor is not played: its outcome is written as -1
// (ongoing) and its length as 0, and the smallest such index is kept
__global__ void hq_count_kernel(const int32_t* desc, long long n, unsigned long long* ctr, int8_t* outcome,
                                int16_t* plies) {
    __shared__ unsigned int hist[kBuckets];
    if (threadIdx.x < kBuckets) hist[threadIdx.x] = 0;
    __syncthreads();
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) {
        const int b = desc_bucket(desc[e]);
        if (b < 0) {
            atomicMin(&ctr[kHostBad], (unsigned long long)e);
            outcome[e] = -1;
            plies[e] = 0;
        } else {
            atomicAdd(&hist[b], 1u);
        }
    }
    __syncthreads();
    if (threadIdx.x < kBuckets && hist[threadIdx.x])
        atomicAdd(&ctr[kHostCount + threadIdx.x], (unsigned long long)hist[threadIdx.x]);
}

// bucket ends = inclusive prefix sums of the counts (one thread: 20 values)
__global__ void hq_scan_kernel(const unsigned long long* ctr, long long* bucket_end) {
    if (threadIdx.x == 0) {
        long long acc = 0;
        for (int b = 0; b < kBuckets; ++b) {
            acc += (long long)ctr[kHostCount + b];
            bucket_end[b] = acc;
        }
    }
}

// queue[begin(b) + k] = the env ids of bucket b (the order inside a bucket
// follows the blocks' reservations; results do not depend on it: every draw
// is keyed by the env's global index)
__global__ void hq_scatter_kernel(const int32_t* desc, long long n, const long long* bucket_end,
                                  unsigned long long* ctr, int32_t* queue) {
    __shared__ unsigned int hist[kBuckets];
    __shared__ unsigned long long base[kBuckets];
    if (threadIdx.x < kBuckets) hist[threadIdx.x] = 0;
    __syncthreads();
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int b = -1;
    unsigned int rank = 0;
    if (e < n) {
        b = desc_bucket(desc[e]);
        if (b >= 0) rank = atomicAdd(&hist[b], 1u);
    }
    __syncthreads();
    if (threadIdx.x < kBuckets && hist[threadIdx.x])
        base[threadIdx.x] = atomicAdd(&ctr[kHostFill + threadIdx.x], (unsigned long long)hist[threadIdx.x]);
    __syncthreads();
    if (b >= 0) queue[(b == 0 ? 0 : bucket_end[b - 1]) + (long long)base[b] + rank] = (int32_t)e;
}
}  // namespace

struct ludax_mixed_plan {
    long long n, env_offset;
    int num_sms;
    ludax_launch_cfg cfg;
    cudaStream_t stream;
    int32_t* d_queue;
    unsigned long long* d_cursor;
    long long bucket_end[kBuckets];
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    cudaGraphNode_t kernel_node;
    cudaKernelNodeParams kparams;
    MixedArgs args;  // kernel parameter block updated before each replay
    // host-buffer path (allocated by its first call)
    uint8_t* d_host;           // descriptors, queue, outcome, plies, counters, bucket ends
    unsigned long long* h_bad;  // pinned: first invalid index of the last host-buffer launch
    bool host_used;
};

extern "C" {

int ludax_rollout_mixed(const int32_t* desc_dev, int64_t num_envs, int64_t env_offset, uint64_t seed,
                        int8_t* outcome_dev, int16_t* plies_dev, const ludax_launch_cfg* cfg, void* stream) {
    ludax::ApiRange api_range("ludax_rollout_mixed");
    if (!desc_dev || !outcome_dev || !plies_dev || num_envs < 1 || num_envs > 0x7FFFFFFFll || env_offset < 0)
        return LUDAX_ERR_ARG;
    if (((uintptr_t)desc_dev % 4) || ((uintptr_t)plies_dev % 2)) return LUDAX_ERR_ALIGN;
    ludax_launch_cfg c = cfg ? *cfg : default_mixed_cfg();
    int st = check_mixed_cfg(c);
    if (st != LUDAX_OK) return st;
    int sms = 0;
    if ((st = num_sms_current(&sms)) != LUDAX_OK) return st;
    std::vector<int32_t> queue;
    MixedArgs a{};
    if ((st = build_queue(desc_dev, num_envs, queue, a.bucket_end, nullptr)) != LUDAX_OK) return st;
    int32_t* d_queue = nullptr;
    unsigned long long* d_cursor = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMalloc(&d_queue, sizeof(int32_t) * num_envs) != cudaSuccess ||
        cudaMalloc(&d_cursor, sizeof(unsigned long long) * kBuckets) != cudaSuccess) {
        cudaFree(d_queue);
        cudaGetLastError();
        return LUDAX_ERR_NOMEM;
    }
    st = LUDAX_OK;
    if (cudaMemcpyAsync(d_queue, queue.data(), sizeof(int32_t) * num_envs, cudaMemcpyHostToDevice, s) != cudaSuccess)
        st = LUDAX_ERR_CUDA;
    a.queue = d_queue;
    a.desc = desc_dev;
    a.n = num_envs;
    a.env_offset = env_offset;
    a.seed_key = splitmix64(seed);
    a.outcome = outcome_dev;
    a.plies = plies_dev;
    a.cursor = d_cursor;
    if (st == LUDAX_OK) st = launch_mixed(a, c, sms, s);
    // the queue and cursor must outlive the launch
    if (cudaStreamSynchronize(s) != cudaSuccess) st = LUDAX_ERR_CUDA;
    cudaFree(d_queue);
    cudaFree(d_cursor);
    return st;
}

int ludax_mixed_plan_create(ludax_mixed_plan** out, const int32_t* desc_dev, int64_t num_envs, int64_t env_offset,
                            const ludax_launch_cfg* cfg, void* stream, int64_t* bad_index) {
    ludax::ApiRange api_range("ludax_mixed_plan_create");
    if (!out || !desc_dev || num_envs < 1 || num_envs > 0x7FFFFFFFll || env_offset < 0) return LUDAX_ERR_ARG;
    *out = nullptr;
    if ((uintptr_t)desc_dev % 4) return LUDAX_ERR_ALIGN;
    ludax_launch_cfg c = cfg ? *cfg : default_mixed_cfg();
    int st = check_mixed_cfg(c);
    if (st != LUDAX_OK) return st;
    ludax_mixed_plan* p = new (std::nothrow) ludax_mixed_plan();
    if (!p) return LUDAX_ERR_NOMEM;
    p->n = num_envs;
    p->env_offset = env_offset;
    p->cfg = c;
    p->stream = (cudaStream_t)stream;
    if ((st = num_sms_current(&p->num_sms)) != LUDAX_OK) {
        delete p;
        return st;
    }
    std::vector<int32_t> queue;
    if ((st = build_queue(desc_dev, num_envs, queue, p->bucket_end, bad_index)) != LUDAX_OK) {
        delete p;
        return st;
    }
    if (cudaMalloc(&p->d_queue, sizeof(int32_t) * num_envs) != cudaSuccess ||
        cudaMalloc(&p->d_cursor, sizeof(unsigned long long) * kBuckets) != cudaSuccess) {
        cudaFree(p->d_queue);
        cudaGetLastError();
        delete p;
        return LUDAX_ERR_NOMEM;
    }
    if (cudaMemcpy(p->d_queue, queue.data(), sizeof(int32_t) * num_envs, cudaMemcpyHostToDevice) != cudaSuccess) {
        ludax_mixed_plan_destroy(p);
        return LUDAX_ERR_CUDA;
    }
    MixedArgs& a = p->args;
    a.queue = p->d_queue;
    a.desc = desc_dev;
    for (int b = 0; b < kBuckets; ++b) a.bucket_end[b] = p->bucket_end[b];
    a.n = num_envs;
    a.env_offset = env_offset;
    a.seed_key = 0;
    a.outcome = nullptr;
    a.plies = nullptr;
    a.cursor = p->d_cursor;
    a.lanes = mixed_lanes(c);  // as launch_mixed sets it (the replays rewrite this parameter block)
    // capture cursor reset + kernel on a private stream
    cudaStream_t cap;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
        ludax_mixed_plan_destroy(p);
        return LUDAX_ERR_CUDA;
    }
    st = LUDAX_OK;
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = LUDAX_ERR_CUDA;
    if (st == LUDAX_OK) {
        int lst = launch_mixed(a, c, p->num_sms, cap);
        cudaError_t e = cudaStreamEndCapture(cap, &p->graph);
        if (lst != LUDAX_OK || e != cudaSuccess) st = LUDAX_ERR_CUDA;
    }
    cudaStreamDestroy(cap);
    if (st == LUDAX_OK) {
        size_t nn = 0;
        cudaGraphGetNodes(p->graph, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        cudaGraphGetNodes(p->graph, nodes.data(), &nn);
        p->kernel_node = nullptr;
        for (auto nd : nodes) {
            cudaGraphNodeType t;
            cudaGraphNodeGetType(nd, &t);
            if (t == cudaGraphNodeTypeKernel) p->kernel_node = nd;
        }
        if (!p->kernel_node || cudaGraphKernelNodeGetParams(p->kernel_node, &p->kparams) != cudaSuccess ||
            cudaGraphInstantiate(&p->exec, p->graph, 0) != cudaSuccess)
            st = LUDAX_ERR_CUDA;
    }
    if (st != LUDAX_OK) {
        cudaGetLastError();
        ludax_mixed_plan_destroy(p);
        return st;
    }
    *out = p;
    return LUDAX_OK;
}

int ludax_mixed_plan_launch(ludax_mixed_plan* p, uint64_t seed, int8_t* outcome_dev, int16_t* plies_dev) {
    ludax::ApiRange api_range("ludax_mixed_plan_launch");
    if (!p || !outcome_dev || !plies_dev) return LUDAX_ERR_ARG;
    if ((uintptr_t)plies_dev % 2) return LUDAX_ERR_ALIGN;
    p->args.seed_key = splitmix64(seed);
    p->args.outcome = outcome_dev;
    p->args.plies = plies_dev;
    void* params[1] = {&p->args};
    cudaKernelNodeParams kp = p->kparams;
    kp.kernelParams = params;
    kp.extra = nullptr;
    if (cudaGraphExecKernelNodeSetParams(p->exec, p->kernel_node, &kp) != cudaSuccess) return LUDAX_ERR_CUDA;
    if (cudaGraphLaunch(p->exec, p->stream) != cudaSuccess) return LUDAX_ERR_CUDA;
    return LUDAX_OK;
}

namespace {
// byte offsets of the host-buffer path's device scratch (each 256-byte aligned)
struct HostLayout {
    size_t desc, queue, out, plies, ctr, end, total;
    explicit HostLayout(long long n) {
        auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
        desc = 0;
        queue = up(desc + 4 * (size_t)n);
        out = up(queue + 4 * (size_t)n);
        plies = up(out + (size_t)n);
        ctr = up(plies + 2 * (size_t)n);
        end = up(ctr + 8 * (size_t)kHostCtrWords);
        total = up(end + 8 * (size_t)kBuckets);
    }
};
}  // namespace

int ludax_mixed_plan_launch_host(ludax_mixed_plan* p, uint64_t seed, const int32_t* desc_host, int8_t* outcome_host,
                                 int16_t* plies_host) {
    ludax::ApiRange api_range("ludax_mixed_plan_launch_host");
    if (!p || !desc_host || !outcome_host || !plies_host) return LUDAX_ERR_ARG;
    const long long n = p->n;
    const HostLayout L(n);
    if (!p->d_host) {
        if (cudaMalloc(&p->d_host, L.total) != cudaSuccess) {
            p->d_host = nullptr;
            cudaGetLastError();
            return LUDAX_ERR_NOMEM;
        }
        if (cudaMallocHost(&p->h_bad, sizeof(unsigned long long)) != cudaSuccess) {
            p->h_bad = nullptr;
            cudaGetLastError();
            return LUDAX_ERR_NOMEM;
        }
    }
    uint8_t* base = p->d_host;
    int32_t* d_desc = reinterpret_cast<int32_t*>(base + L.desc);
    int32_t* d_queue = reinterpret_cast<int32_t*>(base + L.queue);
    int8_t* d_out = reinterpret_cast<int8_t*>(base + L.out);
    int16_t* d_plies = reinterpret_cast<int16_t*>(base + L.plies);
    unsigned long long* d_ctr = reinterpret_cast<unsigned long long*>(base + L.ctr);
    long long* d_end = reinterpret_cast<long long*>(base + L.end);
    cudaStream_t s = p->stream;
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (cudaMemcpyAsync(d_desc, desc_host, 4 * (size_t)n, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return LUDAX_ERR_CUDA;
    hq_init_kernel<<<1, kHostCtrWords, 0, s>>>(d_ctr);
    hq_count_kernel<<<grid, 256, 0, s>>>(d_desc, n, d_ctr, d_out, d_plies);
    hq_scan_kernel<<<1, 32, 0, s>>>(d_ctr, d_end);
    hq_scatter_kernel<<<grid, 256, 0, s>>>(d_desc, n, d_end, d_ctr, d_queue);
    if (cudaGetLastError() != cudaSuccess) return LUDAX_ERR_CUDA;
    MixedArgs a = p->args;
    a.queue = d_queue;
    a.desc = d_desc;
    a.bucket_end_dev = d_end;
    a.seed_key = splitmix64(seed);
    a.outcome = d_out;
    a.plies = d_plies;
    a.cursor = d_ctr;  // words [0, kBuckets): zeroed by launch_mixed
    int st = launch_mixed(a, p->cfg, p->num_sms, s);
    if (st != LUDAX_OK) return st;
    if (cudaMemcpyAsync(outcome_host, d_out, (size_t)n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(plies_host, d_plies, 2 * (size_t)n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(p->h_bad, d_ctr + kHostBad, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess)
        return LUDAX_ERR_CUDA;
    p->host_used = true;
    return LUDAX_OK;
}

int ludax_mixed_plan_sync(ludax_mixed_plan* p, int64_t* bad_index) {
    if (!p) return LUDAX_ERR_ARG;
    if (bad_index) *bad_index = -1;
    if (cudaStreamSynchronize(p->stream) != cudaSuccess) return LUDAX_ERR_CUDA;
    if (!p->host_used || *p->h_bad == ~0ull) return LUDAX_OK;
    const long long e = (long long)*p->h_bad;
    if (bad_index) *bad_index = e;
    int32_t d = 0;
    const int32_t* d_desc = reinterpret_cast<const int32_t*>(p->d_host + HostLayout(p->n).desc);
    if (cudaMemcpyAsync(&d, d_desc + e, sizeof(d), cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
        cudaStreamSynchronize(p->stream) != cudaSuccess)
        return LUDAX_ERR_CUDA;
    return desc_bucket(d) == -2 ? LUDAX_ERR_SIZE : LUDAX_ERR_GAME;
}

int ludax_mixed_plan_destroy(ludax_mixed_plan* p) {
    if (!p) return LUDAX_OK;
    cudaStreamSynchronize(p->stream);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    cudaFree(p->d_queue);
    cudaFree(p->d_cursor);
    cudaFree(p->d_host);
    if (p->h_bad) cudaFreeHost(p->h_bad);
    delete p;
    return cudaGetLastError() == cudaSuccess ? LUDAX_OK : LUDAX_ERR_CUDA;
}

int ludax_autotune_candidates(ludax_launch_cfg* out, int32_t max_out) {
    static const int blocks[] = {64, 128, 192, 256, 384, 448, 512};
    static const int bps[] = {0, 2, 4, 8, 16};
    int k = 0;
    auto put = [&](ludax_launch_cfg c) {
        if (out && k < max_out) out[k] = c;
        ++k;
    };
    for (int t = 0; t < 2; ++t) {
        for (int b : blocks)
            for (int s : bps) {
                if (s > 0 && b * s > 2048) continue;  // more than one SM's threads
                put(ludax_launch_cfg{b, s, 1, t, 0});
            }
        // one thread per env: two envs per thread (the unroll) and part-filled warps (envs per warp)
        for (int b : blocks)
            for (int ept = 1; ept <= 2; ++ept)
                for (int lanes : {32, 16, 8}) {
                    if (ept == 1 && lanes == 32) continue;  // above
                    put(ludax_launch_cfg{b, 0, ept, t, 0, 1, lanes == 32 ? 0 : lanes});
                }
    }
    return k;
}

int ludax_autotune(const int32_t* desc_dev, int64_t num_envs, uint64_t seed, int32_t reps, void* stream,
                   ludax_launch_cfg* best_out, float* best_ms_out, float* ms_table_out, int32_t* n_candidates_out) {
    ludax::ApiRange api_range("ludax_autotune");
    if (!desc_dev || !best_out || num_envs < 1 || reps < 1) return LUDAX_ERR_ARG;
    int nc = ludax_autotune_candidates(nullptr, 0);
    std::vector<ludax_launch_cfg> cands((size_t)nc);
    ludax_autotune_candidates(cands.data(), nc);
    cudaStream_t s = (cudaStream_t)stream;
    int8_t* d_out = nullptr;
    int16_t* d_plies = nullptr;
    if (cudaMalloc(&d_out, num_envs) != cudaSuccess || cudaMalloc(&d_plies, 2 * num_envs) != cudaSuccess) {
        cudaFree(d_out);
        cudaGetLastError();
        return LUDAX_ERR_NOMEM;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int st = LUDAX_OK;
    float best = 1e30f;
    for (int i = 0; i < nc && st == LUDAX_OK; ++i) {
        ludax_mixed_plan* plan = nullptr;
        st = ludax_mixed_plan_create(&plan, desc_dev, num_envs, 0, &cands[(size_t)i], stream, nullptr);
        if (st != LUDAX_OK) break;
        std::vector<float> t;
        for (int r = 0; r < reps + 2 && st == LUDAX_OK; ++r) {
            cudaEventRecord(e0, s);
            st = ludax_mixed_plan_launch(plan, seed + (uint64_t)r, d_out, d_plies);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = LUDAX_ERR_CUDA;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r >= 2) t.push_back(ms);
        }
        ludax_mixed_plan_destroy(plan);
        if (st != LUDAX_OK) break;
        std::sort(t.begin(), t.end());
        float med = t[t.size() / 2];
        if (ms_table_out) ms_table_out[i] = med;
        if (med < best) {
            best = med;
            *best_out = cands[(size_t)i];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d_out);
    cudaFree(d_plies);
    if (best_ms_out) *best_ms_out = best;
    if (n_candidates_out) *n_candidates_out = nc;
    return st;
}

}  // extern "C"

// ===================================================== allocation-free path ==
// ludax_rollout_mixed_noalloc: the same mixed-batch playout as
// ludax_rollout_mixed, for callers that must not allocate device memory --
// a plugin running inside a host framework that owns the device's memory
// budget (its pool has reserved the memory, so a cudaMalloc of ours could
// fail or fragment it), or a serving loop where cudaFree would synchronise
// the device and stall every other stream.  Its scratch (the game-grouped
// work queue and the claim cursors) lives in the static device array below,
// which every GPU that loads this library keeps until the process exits.
namespace {

constexpr long long kNoAllocMaxEnvs = 1ll << 20;  // 4 MiB of queue entries
constexpr int kNoAllocCounterWords = 128;        // cursors, bucket counts and fill positions, first bad index
// layout in 32-bit words: [0, kNoAllocMaxEnvs) queue, then 128 uint64 counters
// (words 0..31 cursors, 32..63 bucket counts, 64..95 fill positions, 96 first bad index)
constexpr int kCtrCount = 32, kCtrPos = 64, kCtrBad = 96;
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocMaxEnvs + 2 * kNoAllocCounterWords];

constexpr int kMaxDevices = 64;
// the array's device address per device, looked up once under the lock
std::atomic<void*> g_noalloc_ptr[kMaxDevices] = {};
std::mutex g_noalloc_mu;

int noalloc_scratch_address(int dev, void** out) {
    void* p = g_noalloc_ptr[dev].load(std::memory_order_acquire);
    if (!p) {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        p = g_noalloc_ptr[dev].load(std::memory_order_relaxed);
        if (!p) {
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return LUDAX_ERR_CUDA;
            }
            g_noalloc_ptr[dev].store(p, std::memory_order_release);
        }
    }
    *out = p;
    return LUDAX_OK;
}

__device__ __forceinline__ int bucket_of_desc_dev(int32_t d) { return desc_bucket(d); }

__global__ void noalloc_reset_kernel(unsigned long long* ctr, long long n) {
    int i = threadIdx.x;
    if (i < kNoAllocCounterWords) ctr[i] = (i == kCtrBad) ? (unsigned long long)n : 0ull;
}

// bucket histogram (block-local, then one atomic per bucket per block) and
// the smallest index of an invalid descriptor
__global__ void noalloc_count_kernel(const int32_t* desc, long long n, unsigned long long* ctr) {
    __shared__ unsigned int hist[kBuckets];
    if (threadIdx.x < kBuckets) hist[threadIdx.x] = 0;
    __syncthreads();
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) {
        int b = bucket_of_desc_dev(desc[e]);
        if (b < 0) atomicMin(&ctr[kCtrBad], (unsigned long long)e);
        else atomicAdd(&hist[b], 1u);
    }
    __syncthreads();
    if (threadIdx.x < kBuckets && hist[threadIdx.x])
        atomicAdd(&ctr[kCtrCount + threadIdx.x], (unsigned long long)hist[threadIdx.x]);
}

struct BucketBegins {
    long long begin[kBuckets];
};

// queue[begin[b] + k] = env ids of bucket b (order inside a bucket follows
// the blocks' reservation order; results do not depend on it)
__global__ void noalloc_scatter_kernel(const int32_t* desc, long long n, BucketBegins bb, unsigned long long* ctr,
                                       int32_t* queue) {
    __shared__ unsigned int hist[kBuckets];
    __shared__ unsigned long long base[kBuckets];
    if (threadIdx.x < kBuckets) hist[threadIdx.x] = 0;
    __syncthreads();
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int b = -1;
    unsigned int rank = 0;
    if (e < n) {
        b = bucket_of_desc_dev(desc[e]);
        if (b >= 0) rank = atomicAdd(&hist[b], 1u);
    }
    __syncthreads();
    if (threadIdx.x < kBuckets && hist[threadIdx.x])
        base[threadIdx.x] = atomicAdd(&ctr[kCtrPos + threadIdx.x], (unsigned long long)hist[threadIdx.x]);
    __syncthreads();
    if (b >= 0) queue[bb.begin[b] + (long long)base[b] + rank] = (int32_t)e;
}

}  // namespace

extern "C" int ludax_rollout_mixed_noalloc(const int32_t* desc_dev, int64_t num_envs, int64_t env_offset, uint64_t seed,
                                           int8_t* outcome_dev, int16_t* plies_dev, const ludax_launch_cfg* cfg,
                                           void* stream, int64_t* bad_index) {
    ludax::ApiRange api_range("ludax_rollout_mixed_noalloc");
    if (!desc_dev || !outcome_dev || !plies_dev || num_envs < 1 || env_offset < 0) return LUDAX_ERR_ARG;
    if (num_envs > kNoAllocMaxEnvs) return LUDAX_ERR_SIZE;  // more envs than the static queue holds
    if (((uintptr_t)desc_dev % 4) || ((uintptr_t)plies_dev % 2)) return LUDAX_ERR_ALIGN;
    ludax_launch_cfg c = cfg ? *cfg : default_mixed_cfg();
    int st = check_mixed_cfg(c);
    if (st != LUDAX_OK) return st;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LUDAX_ERR_CUDA;
    if ((st = num_sms_current(&sms)) != LUDAX_OK) return st;
    // once per device, with that device current: the scratch array's device address
    void* scratch = nullptr;
    if ((st = noalloc_scratch_address(dev, &scratch)) != LUDAX_OK) return st;
    uint32_t* base = static_cast<uint32_t*>(scratch);
    int32_t* queue = reinterpret_cast<int32_t*>(base);
    unsigned long long* ctr = reinterpret_cast<unsigned long long*>(base + kNoAllocMaxEnvs);
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned grid = (unsigned)((num_envs + 255) / 256);
    noalloc_reset_kernel<<<1, kNoAllocCounterWords, 0, s>>>(ctr, num_envs);
    noalloc_count_kernel<<<grid, 256, 0, s>>>(desc_dev, num_envs, ctr);
    unsigned long long h[kNoAllocCounterWords];
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(h, ctr, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return LUDAX_ERR_CUDA;
    if ((long long)h[kCtrBad] < num_envs) {
        long long e = (long long)h[kCtrBad];
        int32_t d = 0;
        if (bad_index) *bad_index = e;
        if (cudaMemcpyAsync(&d, desc_dev + e, sizeof(d), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return LUDAX_ERR_CUDA;
        return bucket_of_desc(d) == -2 ? LUDAX_ERR_SIZE : LUDAX_ERR_GAME;
    }
    if (bad_index) *bad_index = -1;
    BucketBegins bb;
    MixedArgs a{};
    long long acc = 0;
    for (int b = 0; b < kBuckets; ++b) {
        bb.begin[b] = acc;
        acc += (long long)h[kCtrCount + b];
        a.bucket_end[b] = acc;
    }
    noalloc_scatter_kernel<<<grid, 256, 0, s>>>(desc_dev, num_envs, bb, ctr, queue);
    if (cudaGetLastError() != cudaSuccess) return LUDAX_ERR_CUDA;
    a.queue = queue;
    a.desc = desc_dev;
    a.n = num_envs;
    a.env_offset = env_offset;
    a.seed_key = splitmix64(seed);
    a.outcome = outcome_dev;
    a.plies = plies_dev;
    a.cursor = ctr;  // zeroed by launch_mixed before the kernel
    return launch_mixed(a, c, sms, s);
}
