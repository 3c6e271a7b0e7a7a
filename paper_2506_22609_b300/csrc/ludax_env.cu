// ludax_env.cu -- single-game env batches: the C-ABI of include/ludax.h for
// create / reset / legal mask / step / random step / rollout / state view.
//
// Step-per-launch kernels (reset, legal, step, random_step, state view) run
// one thread per env over the structure-of-arrays state in HBM and are bound
// by HBM bandwidth.  ludax_rollout and ludax_rollout_value run one fused
// persistent kernel: each lane keeps an env's bitboards in registers, plays
// it to the end, writes 3 bytes, and claims the next env.
#include <cuda_runtime.h>

#include <chrono>
#include <new>
#include <thread>

#include "../../include/ludax.h"
#include "ludax_hex_lanes.cuh"
#include "ludax_internal.cuh"

using namespace ludax;

namespace {

EnvDev dev_of(const ludax_env* env) {
    return EnvDev{env->d_planes, env->d_meta, env->n, env->env_offset, env->d_counters, env->desc, env->cells};
}

int launch_status() { return cudaGetLastError() == cudaSuccess ? LUDAX_OK : LUDAX_ERR_CUDA; }

unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

// ------------------------------------------------------------- kernels --
template <class G>
__global__ void reset_kernel(EnvDev d, const uint8_t* mask) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= d.n || (mask && !mask[e])) return;
    G g;
    g.reset();
    store_state(g, d, e);
}

template <class G>
__global__ void legal_kernel(EnvDev d, uint64_t* out, uint8_t* pass_legal, int words) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= d.n) return;
    G g;
    set_table(g, nullptr);
    load_state(g, d, e);
    typename G::Mask m{};
    bool pass = false;
    if (g.outcome == kOngoing) {
        m = g.legal();
        pass = G::kHasPass && !any(m);
    }
    if constexpr (IsMove<G>::value) {
        uint64_t* row = out + e * words;
        for (int w = 0; w < words; ++w) row[w] = 0;
        if (g.outcome == kOngoing) g.for_each_move([&](int a) { row[a >> 6] |= 1ull << (a & 63); });
    } else {
        for (int w = 0; w < words; ++w) out[e * words + w] = canon_mask_word(g, m, w);
    }
    if (pass_legal) pass_legal[e] = pass ? 1 : 0;
}

__device__ __forceinline__ float2 rewards_of(int outcome) {
    return outcome == kWin1 ? make_float2(1.f, -1.f) : (outcome == kWin2 ? make_float2(-1.f, 1.f) : make_float2(0.f, 0.f));
}

template <class G>
__global__ void step_kernel(EnvDev d, const int32_t* actions, float2* rewards, uint8_t* terminated) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= d.n) return;
    G g;
    set_table(g, nullptr);
    load_state(g, d, e);
    float2 rw = make_float2(0.f, 0.f);
    if (g.outcome == kOngoing) {
        int a = actions[e];
        typename G::Mask m = g.legal();
        bool ok = false;
        if (G::kHasPass && a == G::kCells) {
            ok = !any(m);
            if (ok) g.pass();
        } else if (a >= 0 && a < actions_of(g) - (G::kHasPass ? 1 : 0)) {
            int b = g.bit_of(a);  // move games: the action's ordinal, -1 if not legal
            ok = b >= 0 && mask_has(m, b);
            if (ok) g.place(b);
        }
        int illegal = 0;
        if (!ok) {
            g.outcome = 2 - g.side;  // the opponent of the mover wins
            illegal = 1;
            atomicAdd(&d.counters[1], 1ull);
        } else if (g.outcome == kOngoing && g.ply >= G::kCap) {
            g.outcome = kCapped;
            atomicAdd(&d.counters[2], 1ull);
        }
        rw = rewards_of(g.outcome);
        store_state(g, d, e, illegal);
    }
    rewards[e] = rw;
    terminated[e] = g.outcome != kOngoing;
}

template <class G>
__global__ void random_step_kernel(EnvDev d, uint64_t seed_key, float2* rewards, uint8_t* terminated) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= d.n) return;
    G g;
    set_table(g, nullptr);
    load_state(g, d, e);
    float2 rw = make_float2(0.f, 0.f);
    if (g.outcome == kOngoing) {
        random_ply(g, env_key(seed_key, (uint64_t)(d.env_offset + e)));
        if (g.outcome == kCapped) atomicAdd(&d.counters[2], 1ull);
        rw = rewards_of(g.outcome);
        store_state(g, d, e);
    }
    rewards[e] = rw;
    terminated[e] = g.outcome != kOngoing;
}

template <class G>
__global__ void get_state_kernel(EnvDev d, ludax_state_view v) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= d.n) return;
    G g;
    set_table(g, nullptr);
    load_state(g, d, e);
    int8_t* b = v.board + e * d.cells;
    if constexpr (IsMove<G>::value) {
        for (int c = 0; c < d.cells; ++c) b[c] = (int8_t)g.cell_value(c);
    } else {
        for (int c = 0; c < d.cells; ++c) {
            int bit = g.bit_of(c);
            int v_own = mask_has(g.own, bit), v_opp = mask_has(g.opp, bit);
            b[c] = (int8_t)(v_own ? g.side + 1 : (v_opp ? 2 - g.side : 0));
        }
    }
    v.to_move[e] = (int8_t)(g.side + 1);
    v.ply[e] = (int16_t)g.ply;
    v.passes[e] = (int8_t)g.passes;
    if constexpr (IsMove<G>::value) v.passes[e] = (int8_t)g.extra();
    if constexpr (G::kGame == Pente::kGame) {  // captured pairs: P1 low nibble, P2 high nibble
        const int c1 = g.side == 0 ? g.caps_own : g.caps_opp, c2 = g.side == 0 ? g.caps_opp : g.caps_own;
        v.passes[e] = (int8_t)((c1 & 15) | ((c2 & 15) << 4));
    }
    v.outcome[e] = (int8_t)g.outcome;
}

template <class M>
__device__ __forceinline__ void set_bit(M& m, int b);
template <>
__device__ __forceinline__ void set_bit<uint32_t>(uint32_t& m, int b) { m |= 1u << b; }
template <>
__device__ __forceinline__ void set_bit<uint64_t>(uint64_t& m, int b) { m |= 1ull << b; }
template <>
__device__ __forceinline__ void set_bit<B128>(B128& m, int b) { m = m | bit128(b); }
template <int W>
__device__ __forceinline__ void set_bit(BitsW<W>& m, int b) { set_bit_w(m, b); }

template <class G>
__global__ void set_state_kernel(EnvDev d, ludax_state_view v) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= d.n) return;
    G g;
    set_table(g, nullptr);
    configure(g, d.desc);
    if constexpr (IsMove<G>::value) {
        g.reset();
        g.clear();
        g.side = v.to_move[e] == 2 ? 1 : 0;  // the pieces are kept relative to the side to move
        const int8_t* b = v.board + e * d.cells;
        for (int c = 0; c < d.cells; ++c) g.set_cell(c, b[c]);
        g.ply = v.ply[e];
        g.passes = 0;
        g.outcome = v.outcome[e];
        g.set_extra((uint8_t)v.passes[e]);
        g.refresh();
        store_state(g, d, e);
    } else {
        typename G::Mask p1{}, p2{};
        const int8_t* b = v.board + e * d.cells;
        for (int c = 0; c < d.cells; ++c) {
            int x = b[c];
            if (x == 1) set_bit(p1, g.bit_of(c));
            if (x == 2) set_bit(p2, g.bit_of(c));
        }
        g.side = v.to_move[e] == 2 ? 1 : 0;
        g.ply = v.ply[e];
        g.passes = v.passes[e];
        g.outcome = v.outcome[e];
        g.own = g.side == 0 ? p1 : p2;
        g.opp = g.side == 0 ? p2 : p1;
        if constexpr (G::kGame == Pente::kGame) {
            const int x = (uint8_t)v.passes[e], c1 = x & 15, c2 = x >> 4;
            g.passes = 0;
            g.caps_own = g.side == 0 ? c1 : c2;
            g.caps_opp = g.side == 0 ? c2 : c1;
        }
        if constexpr (HexN<G>::value != 0) g.rebuild();
        store_state(g, d, e);
    }
}

// ------------------------------------------------- packed state view --
// Per env: V planes (cell value v = 1 .. V; V = 2, or 4 with Draughts'
// kings) of W = ceil(cells / 64) words each in canonical cell order, stored
// plane-major across envs (word w of plane v - 1 of env e at
// planes[((v - 1) * W + w) * n + e]), and one meta word:
// ply | (to_move - 1) << 16 | passes byte << 17 | (outcome + 1) << 25.
__device__ __forceinline__ uint32_t pack_state_meta(int ply, int side, int passes_byte, int outcome) {
    return (uint32_t)(ply & 0xFFFF) | ((uint32_t)(side & 1) << 16) | ((uint32_t)(passes_byte & 0xFF) << 17) |
           ((uint32_t)((outcome + 1) & 7) << 25);
}

template <class G>
__global__ void get_state_bits_kernel(EnvDev d, uint64_t* planes, uint32_t* meta, int W, int V) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= d.n) return;
    G g;
    set_table(g, nullptr);
    load_state(g, d, e);
    int pb = g.passes;
    if constexpr (IsMove<G>::value) {
        for (int v = 1; v <= V; ++v)
            for (int w = 0; w < W; ++w) {
                uint64_t x = 0;
                for (int j = 0; j < 64 && 64 * w + j < d.cells; ++j)
                    if (g.cell_value(64 * w + j) == v) x |= 1ull << j;
                planes[((int64_t)(v - 1) * W + w) * d.n + e] = x;
            }
        pb = g.extra();
    } else {
        const typename G::Mask& p1 = g.side == 0 ? g.own : g.opp;
        const typename G::Mask& p2 = g.side == 0 ? g.opp : g.own;
        for (int w = 0; w < W; ++w) {
            planes[(int64_t)w * d.n + e] = canon_mask_word(g, p1, w);
            planes[(int64_t)(W + w) * d.n + e] = canon_mask_word(g, p2, w);
        }
        if constexpr (G::kGame == Pente::kGame) {
            const int c1 = g.side == 0 ? g.caps_own : g.caps_opp, c2 = g.side == 0 ? g.caps_opp : g.caps_own;
            pb = (c1 & 15) | ((c2 & 15) << 4);
        }
    }
    meta[e] = pack_state_meta(g.ply, g.side, pb, g.outcome);
}

// Builds env e's engine state from the packed view (the state's meta word and
// its V x W plane words); no store.
template <class G>
__device__ __forceinline__ void load_bits(G& g, const EnvDev& d, const uint64_t* planes, const uint32_t* meta,
                                          int64_t e, int W, int V) {
    const uint32_t m = meta[e];
    const int ply = (int)(m & 0xFFFF), side = (int)((m >> 16) & 1), pb = (int)((m >> 17) & 0xFF);
    const int outcome = (int)((m >> 25) & 7) - 1;
    configure(g, d.desc);
    if constexpr (IsMove<G>::value) {
        g.reset();
        g.clear();
        g.side = side;  // the pieces are kept relative to the side to move
        for (int v = 1; v <= V; ++v)
            for (int w = 0; w < W; ++w)
                for (uint64_t x = planes[((int64_t)(v - 1) * W + w) * d.n + e]; x; x &= x - 1) {
                    const int c = 64 * w + __ffsll((long long)x) - 1;
                    if (c < d.cells) g.set_cell(c, v);
                }
        g.ply = ply;
        g.passes = 0;
        g.outcome = outcome;
        g.set_extra(pb);
        g.refresh();
    } else {
        typename G::Mask p1{}, p2{};
        for (int w = 0; w < W; ++w) {
            for (uint64_t x = planes[(int64_t)w * d.n + e]; x; x &= x - 1) {
                const int c = 64 * w + __ffsll((long long)x) - 1;
                if (c < d.cells) set_bit(p1, g.bit_of(c));
            }
            for (uint64_t x = planes[(int64_t)(W + w) * d.n + e]; x; x &= x - 1) {
                const int c = 64 * w + __ffsll((long long)x) - 1;
                if (c < d.cells) set_bit(p2, g.bit_of(c));
            }
        }
        g.side = side;
        g.ply = ply;
        g.passes = pb;
        g.outcome = outcome;
        g.own = side == 0 ? p1 : p2;
        g.opp = side == 0 ? p2 : p1;
        if constexpr (G::kGame == Pente::kGame) {
            g.passes = 0;
            g.caps_own = side == 0 ? (pb & 15) : (pb >> 4);
            g.caps_opp = side == 0 ? (pb >> 4) : (pb & 15);
        }
        if constexpr (HexN<G>::value != 0) g.rebuild();
    }
}

template <class G>
__global__ void set_state_bits_kernel(EnvDev d, const uint64_t* planes, const uint32_t* meta, int W, int V) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= d.n) return;
    G g;
    set_table(g, nullptr);
    load_bits(g, d, planes, meta, e, W, V);
    store_state(g, d, e);
}

// words per plane and planes of the packed state view
void state_bits_shape(const ludax_env* env, int* W, int* V) {
    *W = (env->cells + 63) / 64;
    *V = env->game == LUDAX_GAME_DRAUGHTS ? 4 : 2;
}

// ----------------------------------------------------- fused playouts --
struct RolloutArgs {
    EnvDev d;
    uint64_t seed_key;
    const int16_t* stop;
    int8_t* outcome;
    int16_t* plies;
    int from_start, write_back;
    const uint64_t* bits;        // non-null: start each env from this packed view instead
    const uint32_t* bits_meta;
    int bits_w, bits_v;
    int lanes;                   // rollout_kernel: lanes of each warp that hold envs (1..32)
};

// One persistent kernel: each thread holds EPT envs in registers and advances
// each by one ply per loop trip; a finished env is written out and replaced
// by the next unclaimed env (claim_next).  Work index w < n maps to env w.
// Only the first a.lanes lanes of each warp hold envs (the others leave once
// the block's table is built): slot = warp * a.lanes + lane.
// BITS: the envs start from the packed view in a.bits (the host-buffer path);
// a separate instantiation, so the other launches carry none of its code.
template <class G, int EPT, bool TABLE, bool BITS = false>
__global__ void __launch_bounds__(512) rollout_kernel(RolloutArgs a) {
    extern __shared__ B128 smem_table[];
    const B128* table = nullptr;
    if constexpr (TABLE && HexN<G>::value != 0) {
        hex_fill_table<HexN<G>::value>(smem_table);
        __syncthreads();
        table = smem_table;
    }
    const int64_t n = a.d.n;
    const int lane = threadIdx.x & 31;
    if (lane >= a.lanes) return;
    const int64_t round = (int64_t)gridDim.x * (blockDim.x >> 5) * a.lanes;  // env slots per EPT round
    const int64_t slots = round * EPT;
    const int64_t tid = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * a.lanes + lane;
    const bool refill = slots < n;
    G g[EPT];
    uint64_t key[EPT];
    uint32_t rhi[EPT];
    int stop[EPT];
    int64_t env[EPT];
    bool active[EPT];
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
        env[i] = tid + (int64_t)i * round;
        active[i] = env[i] < n;
        set_table(g[i], table);
    }
    auto init = [&](int i) {
        const int64_t e = env[i];
        configure(g[i], a.d.desc);
        if constexpr (BITS) load_bits(g[i], a.d, a.bits, a.bits_meta, e, a.bits_w, a.bits_v);
        else if (a.from_start) g[i].reset();
        else load_state(g[i], a.d, e);
        key[i] = env_key(a.seed_key, (uint64_t)(a.d.env_offset + e));
        rhi[i] = draw_hi(key[i], (uint32_t)g[i].ply);
        stop[i] = a.stop ? (int)a.stop[e] : 0x7FFF;
    };
#pragma unroll
    for (int i = 0; i < EPT; ++i)
        if (active[i]) init(i);
    for (;;) {
        bool any_active = false;
#pragma unroll
        for (int i = 0; i < EPT; ++i) {
            if (!active[i]) continue;
            any_active = true;
            if (g[i].outcome == kOngoing && g[i].ply < stop[i]) {
                random_ply_pre(g[i], key[i], rhi[i]);
                continue;
            }
            const int64_t e = env[i];
            if (a.outcome) a.outcome[e] = (int8_t)g[i].outcome;
            if (a.plies) a.plies[e] = (int16_t)g[i].ply;
            if (a.write_back) {
                settle_of(g[i]);
                store_state(g[i], a.d, e);
            }
            if (g[i].outcome == kCapped) atomicAdd(&a.d.counters[2], 1ull);
            if (refill) {
                env[i] = slots + claim_next(&a.d.counters[0]);
                active[i] = env[i] < n;
                if (active[i]) init(i);
            } else {
                active[i] = false;
            }
        }
        if (!any_active) break;
    }
}

// Persistent playouts with block-level compaction.  Each round every live env
// plays up to R plies in registers; then the block packs its unfinished envs
// (kWords+2 words each) into shared memory at consecutive slots, so live envs
// occupy the lowest warps and warps with no live env skip the next round's
// plies (they only meet the barriers).  Freed slots take new envs from the
// queue.  Results are independent of the packing: every draw is keyed by
// (seed, global env, ply).
template <class G>
__device__ __forceinline__ void slot_store(uint64_t* buf, int stride, int pos, const G& g, uint64_t key,
                                           long long env, int stop) {
    uint64_t w[G::kWords];
    g.save(w);
#pragma unroll
    for (int i = 0; i < G::kWords; ++i) buf[i * stride + pos] = w[i];
    buf[G::kWords * stride + pos] = key;
    buf[(G::kWords + 1) * stride + pos] = (uint64_t)(uint32_t)env | ((uint64_t)(uint32_t)stop << 32);
}
template <class G>
__device__ __forceinline__ void slot_load(const uint64_t* buf, int stride, int pos, G& g, uint64_t& key,
                                          long long& env, int& stop) {
    uint64_t w[G::kWords];
#pragma unroll
    for (int i = 0; i < G::kWords; ++i) w[i] = buf[i * stride + pos];
    g.load(w);
    key = buf[G::kWords * stride + pos];
    uint64_t x = buf[(G::kWords + 1) * stride + pos];
    env = (long long)(uint32_t)x;
    stop = (int)(x >> 32);
}

template <class G, bool TABLE, bool BITS = false>
__global__ void __launch_bounds__(512) rollout_compact_kernel(RolloutArgs a, int R) {
    extern __shared__ __align__(16) uint64_t smem64[];
    const int B = blockDim.x;
    uint64_t* buf = smem64;                                        // [kWords+2][B]
    int* warp_cnt = reinterpret_cast<int*>(smem64 + (G::kWords + 2) * B);  // [16] + exhausted flag
    const B128* table = nullptr;
    if constexpr (TABLE && HexN<G>::value != 0) {
        B128* t = reinterpret_cast<B128*>(warp_cnt + 32);
        hex_fill_table<HexN<G>::value>(t);
        table = t;
    }
    if (threadIdx.x == 0) warp_cnt[16] = 0;
    __syncthreads();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = B >> 5;
    const long long n = a.d.n;
    const long long slots = (long long)gridDim.x * B;
    const bool refill = slots < n;
    G g;
    set_table(g, table);
    uint64_t key = 0;
    uint32_t rhi = 0;
    long long env = (long long)blockIdx.x * B + tid;
    int stop = 0;
    bool active = env < n;
    auto init = [&]() {
        configure(g, a.d.desc);
        if constexpr (BITS) load_bits(g, a.d, a.bits, a.bits_meta, env, a.bits_w, a.bits_v);
        else if (a.from_start) g.reset();
        else load_state(g, a.d, env);
        key = env_key(a.seed_key, (uint64_t)(a.d.env_offset + env));
        rhi = draw_hi(key, (uint32_t)g.ply);
        stop = a.stop ? (int)a.stop[env] : 0x7FFF;
    };
    if (active) init();
    for (;;) {
        if (active) {
            if constexpr (HexN<G>::value != 0) {
                // two plies per loop body: the six board words that trade roles
                // every ply are renamed instead of moved (Hex 11: ~3% faster;
                // other games measured slower or unchanged)
#pragma unroll 2
                for (int r = 0; r < R; ++r) {
                    if (g.outcome != kOngoing || g.ply >= stop) break;
                    random_ply_pre(g, key, rhi);
                }
            } else {
#pragma unroll 1
                for (int r = 0; r < R; ++r) {
                    if (g.outcome != kOngoing || g.ply >= stop) break;
                    random_ply_pre(g, key, rhi);
                }
            }
            if (g.outcome != kOngoing || g.ply >= stop) {
                if (a.outcome) a.outcome[env] = (int8_t)g.outcome;
                if (a.plies) a.plies[env] = (int16_t)g.ply;
                if (a.write_back) {
                    settle_of(g);
                    store_state(g, a.d, env);
                }
                if (g.outcome == kCapped) atomicAdd(&a.d.counters[2], 1ull);
                active = false;
            }
        }
        const unsigned ball = __ballot_sync(0xFFFFFFFFu, active);
        if (lane == 0) warp_cnt[warp] = __popc(ball);
        __syncthreads();
        int prefix = 0, total = 0;
        for (int w = 0; w < nwarps; ++w) {
            int c = warp_cnt[w];
            prefix += w < warp ? c : 0;
            total += c;
        }
        if (active) slot_store(buf, B, prefix + __popc(ball & ((1u << lane) - 1u)), g, key, env, stop);
        __syncthreads();
        if (tid < total) {
            slot_load(buf, B, tid, g, key, env, stop);
            configure(g, a.d.desc);
            rhi = draw_hi(key, (uint32_t)g.ply);
            active = true;
        } else {
            active = false;
            if (refill && !warp_cnt[16]) {
                env = slots + claim_next(&a.d.counters[0]);
                if (env < n) {
                    init();
                    active = true;
                } else {
                    warp_cnt[16] = 1;  // queue exhausted: stop claiming
                }
            }
        }
        if (!__syncthreads_or(active)) break;
    }
}

// R playouts per env from its stored state; playout j draws with seed + j.
template <class G, bool TABLE>
__global__ void __launch_bounds__(512) rollout_value_kernel(EnvDev d, uint64_t seed, int R, float* value) {
    extern __shared__ B128 smem_table[];
    const B128* table = nullptr;
    if constexpr (TABLE && HexN<G>::value != 0) {
        hex_fill_table<HexN<G>::value>(smem_table);
        __syncthreads();
        table = smem_table;
    }
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= d.n) return;
    G g0, g;
    set_table(g0, table);
    load_state(g0, d, e);
    const uint64_t genv = (uint64_t)(d.env_offset + e);
    float acc = 0.f;
    int j = 0;
    g = g0;
    uint64_t key = env_key(splitmix64(seed), genv);
    uint32_t rhi = draw_hi(key, (uint32_t)g.ply);
    while (j < R) {
        if (g.outcome == kOngoing) {
            random_ply_pre(g, key, rhi);
            continue;
        }
        acc += p1_score(g.outcome);
        ++j;
        g = g0;
        key = env_key(splitmix64(seed + (uint64_t)j), genv);
        rhi = draw_hi(key, (uint32_t)g.ply);
    }
    value[e] = R > 0 ? acc / (float)R : 0.f;
}

// Hex with TPE lanes per env (threads_per_env 2 or 4): a group of TPE
// consecutive lanes plays one env (HexLanes: the board's words split across
// the lanes) and takes the next unclaimed env when its game ends.  Work index
// w < n maps to env w, as in rollout_kernel.
template <int N, int TPE>
__device__ __forceinline__ void load_lanes(HexLanes<N, TPE>& g, const EnvDev& d, int64_t e) {
    int passes;
    unpack_meta(d.meta[e], g.ply, passes, g.side, g.outcome);
    const uint64_t* P = d.planes;
    const int64_t n = d.n;
    const bool p1 = g.side == 0;
    uint32_t s1[HexLanes<N, TPE>::WPL], s2[HexLanes<N, TPE>::WPL], a1[HexLanes<N, TPE>::WPL],
        b1[HexLanes<N, TPE>::WPL], a2[HexLanes<N, TPE>::WPL], b2[HexLanes<N, TPE>::WPL];
    g.words_of(P[0 * n + e], P[1 * n + e], s1);
    g.words_of(P[2 * n + e], P[3 * n + e], s2);
    g.words_of(P[4 * n + e], P[5 * n + e], a1);
    g.words_of(P[6 * n + e], P[7 * n + e], b1);
    g.words_of(P[8 * n + e], P[9 * n + e], a2);
    g.words_of(P[10 * n + e], P[11 * n + e], b2);
#pragma unroll
    for (int j = 0; j < HexLanes<N, TPE>::WPL; ++j) {
        g.own[j] = p1 ? s1[j] : s2[j];
        g.opp[j] = p1 ? s2[j] : s1[j];
        g.ownA[j] = p1 ? a1[j] : a2[j];
        g.ownB[j] = p1 ? b1[j] : b2[j];
        g.oppA[j] = p1 ? a2[j] : a1[j];
        g.oppB[j] = p1 ? b2[j] : b1[j];
        g.front[j] = 0u;
    }
}
template <int N, int TPE>
__device__ __forceinline__ void store_lanes(const HexLanes<N, TPE>& g, const EnvDev& d, int64_t e) {
    const bool p1 = g.side == 0;
    uint64_t w[12];
    w[0] = g.plane_word(p1 ? g.own : g.opp, 0);
    w[1] = g.plane_word(p1 ? g.own : g.opp, 1);
    w[2] = g.plane_word(p1 ? g.opp : g.own, 0);
    w[3] = g.plane_word(p1 ? g.opp : g.own, 1);
    w[4] = g.plane_word(p1 ? g.ownA : g.oppA, 0);
    w[5] = g.plane_word(p1 ? g.ownA : g.oppA, 1);
    w[6] = g.plane_word(p1 ? g.ownB : g.oppB, 0);
    w[7] = g.plane_word(p1 ? g.ownB : g.oppB, 1);
    w[8] = g.plane_word(p1 ? g.oppA : g.ownA, 0);
    w[9] = g.plane_word(p1 ? g.oppA : g.ownA, 1);
    w[10] = g.plane_word(p1 ? g.oppB : g.ownB, 0);
    w[11] = g.plane_word(p1 ? g.oppB : g.ownB, 1);
    if (g.r == 0) {
        d.meta[e] = pack_meta(g.ply, 0, g.side, g.outcome, 0);
#pragma unroll
        for (int k = 0; k < 12; ++k) d.planes[(int64_t)k * d.n + e] = w[k];
    }
}

template <int N, int TPE, bool TABLE>
__global__ void __launch_bounds__(512) rollout_lanes_kernel(RolloutArgs a) {
    __shared__ uint32_t table[TABLE ? N * N * 4 : 1];
    if constexpr (TABLE) {
        for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
            const B128 m = Hex<N>::nbrs(bit128(i));
            table[4 * i + 0] = (uint32_t)m.lo;
            table[4 * i + 1] = (uint32_t)(m.lo >> 32);
            table[4 * i + 2] = (uint32_t)m.hi;
            table[4 * i + 3] = (uint32_t)(m.hi >> 32);
        }
        __syncthreads();
    }
    const int lane = threadIdx.x & 31, r = lane % TPE;
    const unsigned gmask = ((1u << TPE) - 1u) << (lane - r);
    const int64_t n = a.d.n;
    const int64_t groups = (int64_t)gridDim.x * blockDim.x / TPE;
    const bool refill = groups < n;
    HexLanes<N, TPE> g;
    g.init_lane(r, gmask, TABLE ? table : nullptr);
    int64_t env = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / TPE;
    bool active = env < n;
    uint64_t key = 0;
    uint32_t rhi = 0;
    int stop = 0;
    auto init = [&]() {
        if (a.from_start) g.reset();
        else load_lanes(g, a.d, env);
        key = env_key(a.seed_key, (uint64_t)(a.d.env_offset + env));
        rhi = draw_hi(key, (uint32_t)g.ply);
        stop = a.stop ? (int)a.stop[env] : 0x7FFF;
    };
    if (active) init();
    while (active) {  // uniform within a group
        if (g.outcome == kOngoing && g.ply < stop) {
            g.step(key, rhi);
            continue;
        }
        if (a.write_back) {
            g.settle();
            store_lanes(g, a.d, env);
        }
        if (r == 0) {
            if (a.outcome) a.outcome[env] = (int8_t)g.outcome;
            if (a.plies) a.plies[env] = (int16_t)g.ply;
            if (g.outcome == kCapped) atomicAdd(&a.d.counters[2], 1ull);
        }
        if (!refill) break;
        long long next = 0;
        if (r == 0) next = (long long)atomicAdd(&a.d.counters[0], 1ull);
        next = __shfl_sync(gmask, next, lane - r);
        env = groups + next;
        active = env < n;
        if (active) init();
    }
}

template <int N>
int launch_lanes(ludax_env* env, const RolloutArgs& a, const ludax_launch_cfg& cfg) {
    const int block = cfg.block_threads, tpe = cfg.threads_per_env;
    const int64_t per_block = block / tpe;
    int64_t grid = (env->n + per_block - 1) / per_block;
    if (cfg.blocks_per_sm > 0) grid = std::min<int64_t>(grid, (int64_t)env->num_sms * cfg.blocks_per_sm);
    if (grid * per_block < env->n &&
        cudaMemsetAsync(env->d_counters, 0, sizeof(unsigned long long), env->stream) != cudaSuccess)
        return LUDAX_ERR_CUDA;
    const unsigned gd = (unsigned)grid;
    if (tpe == 2) {
        if (cfg.hex_nbr_table) rollout_lanes_kernel<N, 2, true><<<gd, block, 0, env->stream>>>(a);
        else rollout_lanes_kernel<N, 2, false><<<gd, block, 0, env->stream>>>(a);
    } else {
        if (cfg.hex_nbr_table) rollout_lanes_kernel<N, 4, true><<<gd, block, 0, env->stream>>>(a);
        else rollout_lanes_kernel<N, 4, false><<<gd, block, 0, env->stream>>>(a);
    }
    return launch_status();
}

template <class G, bool BITS>
int launch_rollout_as(ludax_env* env, const RolloutArgs& a0, const ludax_launch_cfg& cfg) {
    if constexpr (HexN<G>::value != 0 && !BITS) {
        if (cfg.threads_per_env > 1) return launch_lanes<HexN<G>::value>(env, a0, cfg);
    }
    RolloutArgs a = a0;
    a.lanes = (cfg.lanes_per_warp > 0 && cfg.lanes_per_warp < 32) ? cfg.lanes_per_warp : 32;
    const int block = cfg.block_threads;
    const int ept = BITS ? 1 : cfg.envs_per_thread;  // the packed-view path has one env per thread
    const int64_t per_block = (int64_t)(block / 32) * a.lanes * ept;  // env slots of one block
    int64_t need = (env->n + per_block - 1) / per_block;
    int64_t grid = need;
    if (cfg.blocks_per_sm > 0) {
        int64_t cap = (int64_t)env->num_sms * cfg.blocks_per_sm;
        if (grid > cap) grid = cap;
    }
    const bool table = cfg.hex_nbr_table != 0 && HexN<G>::value != 0;
    size_t smem = table ? sizeof(B128) * G::kCells : 0;
    // the refill cursor is only read when the grid holds fewer slots than envs
    if (grid * per_block < env->n &&
        cudaMemsetAsync(env->d_counters, 0, sizeof(unsigned long long), env->stream) != cudaSuccess)
        return LUDAX_ERR_CUDA;
    if (cfg.compact_every > 0) {
        size_t cs = sizeof(uint64_t) * (G::kWords + 2) * block + 32 * sizeof(int) + smem;
        if (table) {
            auto k = rollout_compact_kernel<G, true, BITS>;
            if (cs > 48 * 1024 && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cs) != cudaSuccess)
                return LUDAX_ERR_CUDA;
            k<<<(unsigned)grid, block, cs, env->stream>>>(a, cfg.compact_every);
        } else {
            auto k = rollout_compact_kernel<G, false, BITS>;
            if (cs > 48 * 1024 && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cs) != cudaSuccess)
                return LUDAX_ERR_CUDA;
            k<<<(unsigned)grid, block, cs, env->stream>>>(a, cfg.compact_every);
        }
        return launch_status();
    }
    if (!BITS && ept == 2) {
        if (table) rollout_kernel<G, 2, true><<<(unsigned)grid, block, smem, env->stream>>>(a);
        else rollout_kernel<G, 2, false><<<(unsigned)grid, block, 0, env->stream>>>(a);
    } else {
        if (table) rollout_kernel<G, 1, true, BITS><<<(unsigned)grid, block, smem, env->stream>>>(a);
        else rollout_kernel<G, 1, false, BITS><<<(unsigned)grid, block, 0, env->stream>>>(a);
    }
    return launch_status();
}

template <class G>
int launch_rollout(ludax_env* env, const RolloutArgs& a, const ludax_launch_cfg& cfg) {
    return a.bits ? launch_rollout_as<G, true>(env, a, cfg) : launch_rollout_as<G, false>(env, a, cfg);
}

ludax_launch_cfg default_cfg() { return ludax_launch_cfg{256, 0, 1, 0, 0}; }

int check_cfg(const ludax_launch_cfg& c) {
    if (c.block_threads < 32 || c.block_threads > 512 || c.block_threads % 32) return LUDAX_ERR_ARG;
    if (c.blocks_per_sm < 0 || c.blocks_per_sm > 64) return LUDAX_ERR_ARG;
    if (c.envs_per_thread != 1 && c.envs_per_thread != 2) return LUDAX_ERR_ARG;
    if (c.hex_nbr_table != 0 && c.hex_nbr_table != 1) return LUDAX_ERR_ARG;
    if (c.compact_every < 0 || c.compact_every > 256) return LUDAX_ERR_ARG;
    if (c.compact_every > 0 && c.envs_per_thread != 1) return LUDAX_ERR_ARG;
    if (c.threads_per_env < 0 || c.threads_per_env == 3 || c.threads_per_env > 4) return LUDAX_ERR_ARG;
    if (c.threads_per_env > 1 && (c.envs_per_thread != 1 || c.compact_every != 0)) return LUDAX_ERR_ARG;
    if (c.lanes_per_warp != 0 && c.lanes_per_warp != 8 && c.lanes_per_warp != 16 && c.lanes_per_warp != 32)
        return LUDAX_ERR_ARG;
    if (c.lanes_per_warp % 32 != 0 && (c.compact_every != 0 || c.threads_per_env > 1)) return LUDAX_ERR_ARG;
    return LUDAX_OK;
}

}  // namespace

// =================================================================== C-ABI ==
extern "C" {

const char* ludax_status_string(int status) {
    switch (status) {
    case LUDAX_OK: return "ok";
    case LUDAX_ERR_ARG: return "invalid argument";
    case LUDAX_ERR_GAME: return "unknown game or descriptor";
    case LUDAX_ERR_SIZE: return "board size not supported for this game";
    case LUDAX_ERR_CUDA: return "CUDA runtime error";
    case LUDAX_ERR_TIMEOUT: return "timed out waiting for the device";
    case LUDAX_ERR_ALIGN: return "misaligned device pointer";
    case LUDAX_ERR_NOMEM: return "device allocation failed";
    default: return "unknown status";
    }
}

int ludax_env_create(ludax_env** out, int32_t game, const ludax_board_params* p, int64_t num_envs, int64_t env_offset,
                     void* stream) {
    if (!out || !p) return LUDAX_ERR_ARG;
    *out = nullptr;
    if (num_envs < 1 || num_envs > 0x7FFFFFFFll || env_offset < 0) return LUDAX_ERR_ARG;
    int planes = 0, cells = 0;
    bool move_game = false;
    int st = dispatch_game(game, p->rows, p->cols, [&](auto tag) {
        using G = typename decltype(tag)::type;
        planes = G::kPlanes;
        cells = G::kGame == LineGame::kGame ? p->rows * p->cols : G::kCells;
        move_game = IsMove<G>::value;
        return LUDAX_OK;
    });
    if (st != LUDAX_OK) return st;
    int32_t desc = game | (p->rows << 8) | (p->cols << 16);
    if (game == LUDAX_GAME_LINE) {
        const int mx = p->rows > p->cols ? p->rows : p->cols;
        if (p->line < 2 || p->line > 15 || p->line > mx || (p->flags & ~7)) return LUDAX_ERR_SIZE;
        desc |= (p->line << 24) | (p->flags << 28);
    } else if (p->line != 0 || p->flags != 0) {
        return LUDAX_ERR_ARG;
    }
    ludax_env* env = new (std::nothrow) ludax_env();
    if (!env) return LUDAX_ERR_NOMEM;
    env->game = game;
    env->rows = p->rows;
    env->cols = p->cols;
    env->cells = cells;
    env->desc = desc;
    env->num_actions = move_game ? env->cells * env->cells : env->cells + (game == LUDAX_GAME_OTHELLO ? 1 : 0);
    env->mask_words = move_game ? (env->num_actions + 63) / 64 : (env->cells + 63) / 64;
    env->planes = planes;
    env->n = num_envs;
    env->env_offset = env_offset;
    env->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&env->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&env->num_sms, cudaDevAttrMultiProcessorCount, env->device) != cudaSuccess) {
        delete env;
        return LUDAX_ERR_CUDA;
    }
    if (cudaMalloc(&env->d_planes, sizeof(uint64_t) * planes * num_envs) != cudaSuccess ||
        cudaMalloc(&env->d_meta, sizeof(uint32_t) * num_envs) != cudaSuccess ||
        cudaMalloc(&env->d_counters, sizeof(unsigned long long) * 4) != cudaSuccess) {
        cudaFree(env->d_planes);
        cudaFree(env->d_meta);
        cudaGetLastError();
        delete env;
        return LUDAX_ERR_NOMEM;
    }
    if (cudaMemsetAsync(env->d_planes, 0, sizeof(uint64_t) * planes * num_envs, env->stream) != cudaSuccess ||
        cudaMemsetAsync(env->d_counters, 0, sizeof(unsigned long long) * 4, env->stream) != cudaSuccess) {
        ludax_env_destroy(env);
        return LUDAX_ERR_CUDA;
    }
    st = ludax_reset(env, nullptr);
    if (st != LUDAX_OK) {
        ludax_env_destroy(env);
        return st;
    }
    *out = env;
    return LUDAX_OK;
}

int ludax_env_destroy(ludax_env* env) {
    if (!env) return LUDAX_OK;
    cudaStreamSynchronize(env->stream);
    cudaFree(env->d_planes);
    cudaFree(env->d_meta);
    cudaFree(env->d_counters);
    cudaFree(env->d_tree);
    cudaFree(env->d_ucb);
    cudaFree(env->d_stage);
    delete env;
    return cudaGetLastError() == cudaSuccess ? LUDAX_OK : LUDAX_ERR_CUDA;
}

int ludax_env_set_stream(ludax_env* env, void* stream) {
    if (!env) return LUDAX_ERR_ARG;
    env->stream = (cudaStream_t)stream;
    return LUDAX_OK;
}

int ludax_env_sizes(const ludax_env* env, int32_t* num_actions, int32_t* mask_words, int64_t* num_envs) {
    if (!env) return LUDAX_ERR_ARG;
    if (num_actions) *num_actions = env->num_actions;
    if (mask_words) *mask_words = env->mask_words;
    if (num_envs) *num_envs = env->n;
    return LUDAX_OK;
}

int ludax_reset(ludax_env* env, const uint8_t* env_mask_dev) {
    ludax::ApiRange api_range("ludax_reset");
    if (!env) return LUDAX_ERR_ARG;
    return dispatch_game(env->game, env->rows, env->cols, [&](auto tag) {
        using G = typename decltype(tag)::type;
        reset_kernel<G><<<grid_for(env->n, 256), 256, 0, env->stream>>>(dev_of(env), env_mask_dev);
        return launch_status();
    });
}

int ludax_legal_mask(ludax_env* env, uint64_t* mask_dev, uint8_t* pass_legal_dev) {
    ludax::ApiRange api_range("ludax_legal_mask");
    if (!env || !mask_dev) return LUDAX_ERR_ARG;
    if (!aligned(mask_dev, 8)) return LUDAX_ERR_ALIGN;
    return dispatch_game(env->game, env->rows, env->cols, [&](auto tag) {
        using G = typename decltype(tag)::type;
        legal_kernel<G><<<grid_for(env->n, 256), 256, 0, env->stream>>>(dev_of(env), mask_dev, pass_legal_dev,
                                                                           env->mask_words);
        return launch_status();
    });
}

int ludax_step(ludax_env* env, const int32_t* actions_dev, float* rewards_dev, uint8_t* terminated_dev) {
    ludax::ApiRange api_range("ludax_step");
    if (!env || !actions_dev || !rewards_dev || !terminated_dev) return LUDAX_ERR_ARG;
    if (!aligned(actions_dev, 4) || !aligned(rewards_dev, 8)) return LUDAX_ERR_ALIGN;
    return dispatch_game(env->game, env->rows, env->cols, [&](auto tag) {
        using G = typename decltype(tag)::type;
        step_kernel<G><<<grid_for(env->n, 256), 256, 0, env->stream>>>(dev_of(env), actions_dev,
                                                                          (float2*)rewards_dev, terminated_dev);
        return launch_status();
    });
}

int ludax_random_step(ludax_env* env, uint64_t seed, float* rewards_dev, uint8_t* terminated_dev) {
    ludax::ApiRange api_range("ludax_random_step");
    if (!env || !rewards_dev || !terminated_dev) return LUDAX_ERR_ARG;
    if (!aligned(rewards_dev, 8)) return LUDAX_ERR_ALIGN;
    return dispatch_game(env->game, env->rows, env->cols, [&](auto tag) {
        using G = typename decltype(tag)::type;
        random_step_kernel<G><<<grid_for(env->n, 256), 256, 0, env->stream>>>(dev_of(env), splitmix64(seed),
                                                                                 (float2*)rewards_dev, terminated_dev);
        return launch_status();
    });
}

// the playouts of ludax_rollout; with bits non-null every env starts from the
// packed view (bits, bits_meta) instead of its stored or start state
static int rollout_impl(ludax_env* env, uint64_t seed, uint32_t flags, const int16_t* stop_ply_dev,
                        int8_t* outcome_dev, int16_t* plies_dev, const ludax_launch_cfg* cfg, const uint64_t* bits,
                        const uint32_t* bits_meta) {
    if (!env) return LUDAX_ERR_ARG;
    if (flags & ~(uint32_t)(LUDAX_ROLLOUT_FROM_START | LUDAX_ROLLOUT_WRITE_BACK)) return LUDAX_ERR_ARG;
    if ((stop_ply_dev && !aligned(stop_ply_dev, 2)) || (plies_dev && !aligned(plies_dev, 2))) return LUDAX_ERR_ALIGN;
    ludax_launch_cfg c = cfg ? *cfg : default_cfg();
    int st = check_cfg(c);
    if (st != LUDAX_OK) return st;
    // several lanes per env: Hex playouts from the env's own or start state only
    if (c.threads_per_env > 1 && (env->game != LUDAX_GAME_HEX || bits)) return LUDAX_ERR_ARG;
    RolloutArgs a;
    a.d = dev_of(env);
    a.seed_key = splitmix64(seed);
    a.stop = stop_ply_dev;
    a.outcome = outcome_dev;
    a.plies = plies_dev;
    a.from_start = (flags & LUDAX_ROLLOUT_FROM_START) ? 1 : 0;
    a.write_back = (flags & LUDAX_ROLLOUT_WRITE_BACK) ? 1 : 0;
    a.bits = bits;
    a.bits_meta = bits_meta;
    state_bits_shape(env, &a.bits_w, &a.bits_v);
    return dispatch_game(env->game, env->rows, env->cols, [&](auto tag) {
        using G = typename decltype(tag)::type;
        return launch_rollout<G>(env, a, c);
    });
}

int ludax_rollout(ludax_env* env, uint64_t seed, uint32_t flags, const int16_t* stop_ply_dev, int8_t* outcome_dev,
                  int16_t* plies_dev, const ludax_launch_cfg* cfg) {
    ludax::ApiRange api_range("ludax_rollout");
    return rollout_impl(env, seed, flags, stop_ply_dev, outcome_dev, plies_dev, cfg, nullptr, nullptr);
}

// device staging of the host-buffer playouts: planes, meta, outcome, plies
static int host_stage(ludax_env* env, size_t pbytes, size_t* out_at, size_t* plies_at) {
    const size_t n = (size_t)env->n;
    *out_at = pbytes + 4 * n;
    *plies_at = *out_at + n + (n & 1);
    const size_t need = *plies_at + 2 * n;
    if (env->stage_bytes < need) {
        if (cudaStreamSynchronize(env->stream) != cudaSuccess) return LUDAX_ERR_CUDA;  // a previous call may still use it
        cudaFree(env->d_stage);
        env->d_stage = nullptr;
        env->stage_bytes = 0;
        if (cudaMalloc(&env->d_stage, need) != cudaSuccess) {
            cudaGetLastError();
            return LUDAX_ERR_NOMEM;
        }
        env->stage_bytes = need;
    }
    return LUDAX_OK;
}

int ludax_rollout_host(ludax_env* env, const uint64_t* planes_host, const uint32_t* meta_host, uint64_t seed,
                       int8_t* outcome_host, int16_t* plies_host, const ludax_launch_cfg* cfg) {
    ludax::ApiRange api_range("ludax_rollout_host");
    if (!env || !planes_host || !meta_host || !outcome_host || !plies_host) return LUDAX_ERR_ARG;
    int W, V;
    state_bits_shape(env, &W, &V);
    const size_t n = (size_t)env->n, pbytes = (size_t)W * V * n * 8;
    size_t out_at, plies_at;
    int st = host_stage(env, pbytes, &out_at, &plies_at);
    if (st) return st;
    uint64_t* dp = reinterpret_cast<uint64_t*>(env->d_stage);
    uint32_t* dm = reinterpret_cast<uint32_t*>(env->d_stage + pbytes);
    int8_t* dout = reinterpret_cast<int8_t*>(env->d_stage + out_at);
    int16_t* dpl = reinterpret_cast<int16_t*>(env->d_stage + plies_at);
    if (cudaMemcpyAsync(dp, planes_host, pbytes, cudaMemcpyHostToDevice, env->stream) != cudaSuccess ||
        cudaMemcpyAsync(dm, meta_host, 4 * n, cudaMemcpyHostToDevice, env->stream) != cudaSuccess)
        return LUDAX_ERR_CUDA;
    // the playouts load the packed positions themselves (no separate load launch)
    if ((st = rollout_impl(env, seed, 0, nullptr, dout, dpl, cfg, dp, dm))) return st;
    if (cudaMemcpyAsync(outcome_host, dout, n, cudaMemcpyDeviceToHost, env->stream) != cudaSuccess ||
        cudaMemcpyAsync(plies_host, dpl, 2 * n, cudaMemcpyDeviceToHost, env->stream) != cudaSuccess)
        return LUDAX_ERR_CUDA;
    return LUDAX_OK;
}

int ludax_rollout_host_packed(ludax_env* env, const void* in_host, void* out_host, uint64_t seed,
                              const ludax_launch_cfg* cfg) {
    ludax::ApiRange api_range("ludax_rollout_host_packed");
    if (!env || !in_host || !out_host) return LUDAX_ERR_ARG;
    int W, V;
    state_bits_shape(env, &W, &V);
    const size_t n = (size_t)env->n, pbytes = (size_t)W * V * n * 8;
    size_t out_at, plies_at;
    int st = host_stage(env, pbytes, &out_at, &plies_at);
    if (st) return st;
    uint64_t* dp = reinterpret_cast<uint64_t*>(env->d_stage);
    uint32_t* dm = reinterpret_cast<uint32_t*>(env->d_stage + pbytes);
    int8_t* dout = reinterpret_cast<int8_t*>(env->d_stage + out_at);
    int16_t* dpl = reinterpret_cast<int16_t*>(env->d_stage + plies_at);
    if (cudaMemcpyAsync(dp, in_host, out_at, cudaMemcpyHostToDevice, env->stream) != cudaSuccess) return LUDAX_ERR_CUDA;
    if ((st = rollout_impl(env, seed, 0, nullptr, dout, dpl, cfg, dp, dm))) return st;
    if (cudaMemcpyAsync(out_host, dout, plies_at + 2 * n - out_at, cudaMemcpyDeviceToHost, env->stream) != cudaSuccess)
        return LUDAX_ERR_CUDA;
    return LUDAX_OK;
}

int ludax_rollout_value(ludax_env* env, uint64_t seed, int32_t R, float* value_dev, const ludax_launch_cfg* cfg) {
    ludax::ApiRange api_range("ludax_rollout_value");
    if (!env || !value_dev || R < 1) return LUDAX_ERR_ARG;
    if (!aligned(value_dev, 4)) return LUDAX_ERR_ALIGN;
    ludax_launch_cfg c = cfg ? *cfg : default_cfg();
    int st = check_cfg(c);
    if (st != LUDAX_OK) return st;
    if (c.threads_per_env > 1 || c.lanes_per_warp % 32 != 0) return LUDAX_ERR_ARG;  // one lane per env, full warps
    return dispatch_game(env->game, env->rows, env->cols, [&](auto tag) {
        using G = typename decltype(tag)::type;
        const bool table = c.hex_nbr_table != 0 && HexN<G>::value != 0;
        size_t smem = table ? sizeof(B128) * G::kCells : 0;
        unsigned grid = grid_for(env->n, c.block_threads);
        if (table)
            rollout_value_kernel<G, true><<<grid, c.block_threads, smem, env->stream>>>(dev_of(env), seed, R, value_dev);
        else
            rollout_value_kernel<G, false><<<grid, c.block_threads, 0, env->stream>>>(dev_of(env), seed, R, value_dev);
        return launch_status();
    });
}

int ludax_get_state(ludax_env* env, const ludax_state_view* dst) {
    ludax::ApiRange api_range("ludax_get_state");
    if (!env || !dst || !dst->board || !dst->to_move || !dst->ply || !dst->passes || !dst->outcome) return LUDAX_ERR_ARG;
    if (!aligned(dst->ply, 2)) return LUDAX_ERR_ALIGN;
    ludax_state_view v = *dst;
    return dispatch_game(env->game, env->rows, env->cols, [&](auto tag) {
        using G = typename decltype(tag)::type;
        get_state_kernel<G><<<grid_for(env->n, 128), 128, 0, env->stream>>>(dev_of(env), v);
        return launch_status();
    });
}

int ludax_set_state(ludax_env* env, const ludax_state_view* src) {
    ludax::ApiRange api_range("ludax_set_state");
    if (!env || !src || !src->board || !src->to_move || !src->ply || !src->passes || !src->outcome) return LUDAX_ERR_ARG;
    if (!aligned(src->ply, 2)) return LUDAX_ERR_ALIGN;
    ludax_state_view v = *src;
    return dispatch_game(env->game, env->rows, env->cols, [&](auto tag) {
        using G = typename decltype(tag)::type;
        set_state_kernel<G><<<grid_for(env->n, 128), 128, 0, env->stream>>>(dev_of(env), v);
        return launch_status();
    });
}

int ludax_state_bits_words(const ludax_env* env, int32_t* words_per_env) {
    if (!env || !words_per_env) return LUDAX_ERR_ARG;
    int W, V;
    state_bits_shape(env, &W, &V);
    *words_per_env = W * V;
    return LUDAX_OK;
}

int ludax_get_state_bits(ludax_env* env, uint64_t* planes_dev, uint32_t* meta_dev) {
    ludax::ApiRange api_range("ludax_get_state_bits");
    if (!env || !planes_dev || !meta_dev) return LUDAX_ERR_ARG;
    if (!aligned(planes_dev, 8) || !aligned(meta_dev, 4)) return LUDAX_ERR_ALIGN;
    int W, V;
    state_bits_shape(env, &W, &V);
    return dispatch_game(env->game, env->rows, env->cols, [&](auto tag) {
        using G = typename decltype(tag)::type;
        get_state_bits_kernel<G><<<grid_for(env->n, 128), 128, 0, env->stream>>>(dev_of(env), planes_dev, meta_dev, W, V);
        return launch_status();
    });
}

int ludax_set_state_bits(ludax_env* env, const uint64_t* planes_dev, const uint32_t* meta_dev) {
    ludax::ApiRange api_range("ludax_set_state_bits");
    if (!env || !planes_dev || !meta_dev) return LUDAX_ERR_ARG;
    if (!aligned(planes_dev, 8) || !aligned(meta_dev, 4)) return LUDAX_ERR_ALIGN;
    int W, V;
    state_bits_shape(env, &W, &V);
    return dispatch_game(env->game, env->rows, env->cols, [&](auto tag) {
        using G = typename decltype(tag)::type;
        set_state_bits_kernel<G><<<grid_for(env->n, 128), 128, 0, env->stream>>>(dev_of(env), planes_dev, meta_dev, W, V);
        return launch_status();
    });
}

int ludax_counters(ludax_env* env, int64_t* illegal_actions, int64_t* capped) {
    if (!env) return LUDAX_ERR_ARG;
    unsigned long long h[4];
    if (cudaMemcpyAsync(h, env->d_counters, sizeof(h), cudaMemcpyDeviceToHost, env->stream) != cudaSuccess ||
        cudaStreamSynchronize(env->stream) != cudaSuccess)
        return LUDAX_ERR_CUDA;
    if (illegal_actions) *illegal_actions = (int64_t)h[1];
    if (capped) *capped = (int64_t)h[2];
    return LUDAX_OK;
}

int ludax_sync(ludax_env* env, int64_t timeout_ms) {
    if (!env) return LUDAX_ERR_ARG;
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t q = cudaStreamQuery(env->stream);
        if (q == cudaSuccess) return LUDAX_OK;
        if (q != cudaErrorNotReady) return LUDAX_ERR_CUDA;
        if (timeout_ms >= 0) {
            auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0);
            if (ms.count() >= timeout_ms) return LUDAX_ERR_TIMEOUT;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

int ludax_autotune_env_candidates(const ludax_env* env, ludax_launch_cfg* out, int32_t max_out) {
    if (!env) return LUDAX_ERR_ARG;
    static const int blocks[] = {64, 128, 192, 256, 384, 448, 512};
    static const int bps[] = {0, 2, 4, 8, 16};
    static const int compacts[] = {0, 4, 8, 16};
    const bool hex = env->game == LUDAX_GAME_HEX;
    int k = 0;
    auto put = [&](ludax_launch_cfg c) {
        if (out && k < max_out) out[k] = c;
        ++k;
    };
    for (int t = 0; t < (hex ? 2 : 1); ++t) {
        for (int ce : compacts)
            for (int ept = 1; ept <= 2; ++ept)
                for (int b : blocks)
                    for (int s : bps) {
                        if (s > 0 && b * s > 2048) continue;
                        if (ce > 0 && ept != 1) continue;
                        put(ludax_launch_cfg{b, s, ept, t, ce, 1});
                    }
        // part-filled warps (one thread per env, no persistence): for small batches
        for (int lanes : {8, 16})
            for (int ept = 1; ept <= 2; ++ept)
                for (int b : blocks) put(ludax_launch_cfg{b, 0, ept, t, 0, 1, lanes});
        if (hex)  // several lanes per env
            for (int tpe : {2, 4})
                for (int b : blocks)
                    for (int s : bps) {
                        if (s > 0 && b * s > 2048) continue;
                        put(ludax_launch_cfg{b, s, 1, t, 0, tpe});
                    }
    }
    return k;
}

int ludax_autotune_env(ludax_env* env, uint64_t seed, int32_t reps, ludax_launch_cfg* best_out, float* best_ms_out,
                       float* ms_table_out, int32_t* n_candidates_out) {
    ludax::ApiRange api_range("ludax_autotune_env");
    if (!env || !best_out || reps < 1) return LUDAX_ERR_ARG;
    const int nc = ludax_autotune_env_candidates(env, nullptr, 0);
    ludax_launch_cfg* cands = new (std::nothrow) ludax_launch_cfg[(size_t)nc];
    if (!cands) return LUDAX_ERR_NOMEM;
    ludax_autotune_env_candidates(env, cands, nc);
    int8_t* d_out = nullptr;
    int16_t* d_plies = nullptr;
    if (cudaMalloc(&d_out, env->n) != cudaSuccess || cudaMalloc(&d_plies, 2 * env->n) != cudaSuccess) {
        cudaFree(d_out);
        cudaGetLastError();
        delete[] cands;
        return LUDAX_ERR_NOMEM;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int st = LUDAX_OK, k = 0;
    float best = 1e30f;
    for (int i = 0; i < nc && st == LUDAX_OK; ++i) {
        const ludax_launch_cfg c = cands[i];
        float ts[64];
        int nt = 0;
        for (int r = 0; r < reps + 2 && st == LUDAX_OK; ++r) {
            cudaEventRecord(e0, env->stream);
            st = ludax_rollout(env, seed + (uint64_t)r, LUDAX_ROLLOUT_FROM_START, nullptr, d_out, d_plies, &c);
            cudaEventRecord(e1, env->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = LUDAX_ERR_CUDA;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r >= 2 && nt < 64) ts[nt++] = ms;
        }
        if (st != LUDAX_OK) break;
        for (int a = 1; a < nt; ++a)
            for (int j = a; j > 0 && ts[j] < ts[j - 1]; --j) {
                float x = ts[j]; ts[j] = ts[j - 1]; ts[j - 1] = x;
            }
        const float med = ts[nt / 2];
        if (ms_table_out && k < 512) ms_table_out[k] = med;
        ++k;
        if (med < best) {
            best = med;
            *best_out = c;
        }
    }
    delete[] cands;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d_out);
    cudaFree(d_plies);
    if (best_ms_out) *best_ms_out = best;
    if (n_candidates_out) *n_candidates_out = k;
    return st;
}

}  // extern "C"
