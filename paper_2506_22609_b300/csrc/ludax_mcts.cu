// ludax_mcts.cu -- UCT agents (MCTS with the UCB1 rule and a uniform-random
// playout at each new leaf) and whole agent-vs-agent matches, the agents of
// the GAVEL-like evaluation in App. F ("MCTS with UCB1", a number of
// iterations per move, each a traversal, an expansion and a random rollout).
//
// One thread owns one search (or one match, whose searches it runs one after
// the other).  The game state lives in registers and is re-derived along the
// path from the root at every iteration; the tree lives in a per-env slab of
// the env's scratch buffer: 16-byte nodes {parent, action, first child, next
// sibling, N, W} and one tried-action bitboard per node.  Rewards are integer
// half points (win 2, draw 1, loss 0), so back-propagation is exact and the
// UCB1 score W/(2N) + T[N_parent]/sqrt(N) is computed with correctly rounded
// double division and square root; T[m] = c*sqrt(ln m) is tabulated on the
// host.  Every loop is bounded by the iteration count and the game's ply cap.
#include <cmath>
#include <vector>

#include "ludax_internal.cuh"

namespace {
using namespace ludax;

struct TNode {
    int16_t parent, action, first_child, next_sibling;  // action: internal bit, -1 = pass
    uint32_t N, W;
};
static_assert(sizeof(TNode) == 16, "tree node is 16 bytes");

// 64-bit words of a legal-action mask
template <class M>
struct MaskWords;
template <>
struct MaskWords<uint32_t> {
    static constexpr int value = 1;
};
template <>
struct MaskWords<uint64_t> {
    static constexpr int value = 1;
};
template <>
struct MaskWords<B128> {
    static constexpr int value = 2;
};
template <int W>
struct MaskWords<BitsW<W>> {
    static constexpr int value = W;
};

__device__ __forceinline__ void mask_put(uint64_t* p, uint32_t m) { p[0] = m; }
__device__ __forceinline__ void mask_put(uint64_t* p, uint64_t m) { p[0] = m; }
__device__ __forceinline__ void mask_put(uint64_t* p, B128 m) {
    p[0] = m.lo;
    p[1] = m.hi;
}
template <int W>
__device__ __forceinline__ void mask_put(uint64_t* p, const BitsW<W>& m) {
#pragma unroll
    for (int i = 0; i < W; ++i) p[i] = m.w[i];
}
__device__ __forceinline__ void mask_get(const uint64_t* p, uint32_t& m) { m = (uint32_t)p[0]; }
__device__ __forceinline__ void mask_get(const uint64_t* p, uint64_t& m) { m = p[0]; }
__device__ __forceinline__ void mask_get(const uint64_t* p, B128& m) { m = B128{p[0], p[1]}; }
template <int W>
__device__ __forceinline__ void mask_get(const uint64_t* p, BitsW<W>& m) {
#pragma unroll
    for (int i = 0; i < W; ++i) m.w[i] = p[i];
}
__device__ __forceinline__ void mask_zero(uint64_t* p, int words) {
    for (int i = 0; i < words; ++i) p[i] = 0;
}
__device__ __forceinline__ void mask_add(uint32_t& m, int b) { m |= 1u << b; }
__device__ __forceinline__ void mask_add(uint64_t& m, int b) { m |= 1ull << b; }
__device__ __forceinline__ void mask_add(B128& m, int b) { m = m | bit128(b); }
template <int W>
__device__ __forceinline__ void mask_add(BitsW<W>& m, int b) {
    set_bit_w(m, b);
}

template <class G>
__device__ __forceinline__ void play(G& g, int action) {
    if (action < 0) g.pass();
    else g.place(action);
    if (g.outcome == kOngoing && g.ply >= G::kCap) g.outcome = kCapped;
}

// half points for the side `mover` (0 = P1) from a final outcome
__device__ __forceinline__ uint32_t half_points(int outcome, int mover) {
    if (outcome == mover + 1) return 2u;
    return (outcome == kDraw || outcome == kCapped) ? 1u : 0u;
}

__device__ __forceinline__ double ucb1(uint32_t W, uint32_t N, double t) {
    const double n = (double)N;
    return __dadd_rn(__ddiv_rn((double)W, __dmul_rn(2.0, n)), __ddiv_rn(t, __dsqrt_rn(n)));
}

// One search from `root`; returns the chosen action (internal bit, -1 = pass).
// nd / mk: this thread's node slab and tried masks (iters + 1 nodes).
template <class G>
__device__ int uct_search(const G& root, uint64_t key, int iters, const double* __restrict__ T, TNode* nd,
                          uint64_t* mk) {
    using M = typename G::Mask;
    constexpr int MW = MaskWords<M>::value;
    nd[0] = TNode{-1, -1, -1, -1, 0u, 0u};
    mask_zero(mk, MW);
    int count = 1;
    const int side0 = root.side;
    for (int i = 0; i < iters; ++i) {
        const uint64_t ki = splitmix64(key ^ (uint64_t)i);
        G g = root;
        int x = 0, depth = 0;
        while (g.outcome == kOngoing) {
            const M legal = g.legal();
            if (G::kHasPass && !any(legal)) {  // the forced pass is the only action
                if (nd[x].first_child < 0) {
                    const int y = count++;
                    nd[y] = TNode{(int16_t)x, -1, -1, -1, 0u, 0u};
                    mask_zero(mk + (size_t)y * MW, MW);
                    nd[x].first_child = (int16_t)y;
                    play(g, -1);
                    x = y;
                    ++depth;
                    break;
                }
                x = nd[x].first_child;
                play(g, -1);
                ++depth;
                continue;
            }
            M tried;
            mask_get(mk + (size_t)x * MW, tried);
            const M untried = legal & ~tried;
            if (any(untried)) {
                const uint32_t k = __umulhi((uint32_t)(splitmix64(~ki) >> 32), popc(untried));
                const int b = select_bit(untried, k);
                mask_add(tried, b);
                mask_put(mk + (size_t)x * MW, tried);
                const int y = count++;
                nd[y] = TNode{(int16_t)x, (int16_t)b, -1, nd[x].first_child, 0u, 0u};
                mask_zero(mk + (size_t)y * MW, MW);
                nd[x].first_child = (int16_t)y;
                play(g, b);
                x = y;
                ++depth;
                break;
            }
            // every legal action has a child: UCB1, the smallest action on a tie
            const double t = T[nd[x].N];
            int best = -1, best_a = 0;
            double bq = 0.0;
            for (int y = nd[x].first_child; y >= 0; y = nd[y].next_sibling) {
                const TNode c = nd[y];
                const double q = ucb1(c.W, c.N, t);
                if (best < 0 || q > bq || (q == bq && c.action < best_a)) {
                    best = y;
                    bq = q;
                    best_a = c.action;
                }
            }
            play(g, best_a);
            x = best;
            ++depth;
        }
        while (g.outcome == kOngoing) random_ply(g, ki);
        // every ply alternates the side to move, so the node at depth d was
        // entered by side (side0 + d - 1) mod 2
        for (int y = x, d = depth; y > 0; y = nd[y].parent, --d) {
            nd[y].N += 1u;
            nd[y].W += half_points(g.outcome, (side0 + d - 1) & 1);
        }
        nd[0].N += 1u;
    }
    int best = -1;
    for (int y = nd[0].first_child; y >= 0; y = nd[y].next_sibling) {
        if (best < 0) {
            best = y;
            continue;
        }
        const TNode c = nd[y], b = nd[best];
        if (c.N > b.N || (c.N == b.N && (c.W > b.W || (c.W == b.W && c.action < b.action)))) best = y;
    }
    return best < 0 ? -1 : nd[best].action;
}

__device__ __forceinline__ uint64_t search_key(uint64_t seed_key, int64_t match, int ply) {
    return splitmix64(env_key(seed_key, (uint64_t)match) ^ ((uint64_t)(ply + 1) << 32));
}

struct MctsArgs {
    EnvDev d;
    uint64_t seed_key;  // splitmix64(seed)
    int iters_p1, iters_p2, cap_nodes, num_actions;
    const double* T;
    TNode* nodes;
    uint64_t* masks;
    // search mode
    int32_t* action;
    uint32_t* visits;
    uint32_t* wins;
    // match mode
    int from_start, write_back;
    int8_t* outcome;
    int16_t* plies;
    int16_t* agency;
    int16_t* coverage;
};

template <class G>
__global__ void __launch_bounds__(128) uct_search_kernel(MctsArgs a) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.d.n) return;
    constexpr int MW = MaskWords<typename G::Mask>::value;
    TNode* nd = a.nodes + (size_t)e * a.cap_nodes;
    uint64_t* mk = a.masks + (size_t)e * a.cap_nodes * MW;
    G g;
    set_table(g, nullptr);
    load_state(g, a.d, e);
    int act = -1;
    if (g.outcome == kOngoing) {
        const int b = uct_search(g, search_key(a.seed_key, a.d.env_offset + e, g.ply), a.iters_p1, a.T, nd, mk);
        act = b < 0 ? G::kCells : g.canon_of(b);
    }
    a.action[e] = act;
    if (a.visits || a.wins) {
        const size_t row = (size_t)e * a.num_actions;
        for (int j = 0; j < a.num_actions; ++j) {
            if (a.visits) a.visits[row + j] = 0u;
            if (a.wins) a.wins[row + j] = 0u;
        }
        if (act >= 0) {
            for (int y = nd[0].first_child; y >= 0; y = nd[y].next_sibling) {
                const int j = nd[y].action < 0 ? G::kCells : g.canon_of(nd[y].action);
                if (a.visits) a.visits[row + j] = nd[y].N;
                if (a.wins) a.wins[row + j] = nd[y].W;
            }
        }
    }
}

template <class G>
__global__ void __launch_bounds__(128) uct_match_kernel(MctsArgs a) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.d.n) return;
    constexpr int MW = MaskWords<typename G::Mask>::value;
    TNode* nd = a.nodes + (size_t)e * a.cap_nodes;
    uint64_t* mk = a.masks + (size_t)e * a.cap_nodes * MW;
    G g;
    set_table(g, nullptr);
    if (a.from_start) {
        configure(g, a.d.desc);
        g.reset();
    } else {
        load_state(g, a.d, e);
    }
    const int64_t match = a.d.env_offset + e;
    typename G::Mask ever = g.own | g.opp;
    int turns = 0;
    while (g.outcome == kOngoing) {
        const typename G::Mask legal = g.legal();
        int b = -1;
        if (!(G::kHasPass && !any(legal))) {
            if (popc(legal) > 1) {
                ++turns;
                b = uct_search(g, search_key(a.seed_key, match, g.ply), g.side == 0 ? a.iters_p1 : a.iters_p2, a.T,
                               nd, mk);
            } else {
                b = select_bit(legal, 0u);
            }
        }
        play(g, b);
        ever = ever | g.own | g.opp;
    }
    if (a.outcome) a.outcome[e] = (int8_t)g.outcome;
    if (a.plies) a.plies[e] = (int16_t)g.ply;
    if (a.agency) a.agency[e] = (int16_t)turns;
    if (a.coverage) a.coverage[e] = (int16_t)popc(ever);
    if (a.write_back) store_state(g, a.d, e);
}

EnvDev dev_of(const ludax_env* env) {
    return EnvDev{env->d_planes, env->d_meta, env->n, env->env_offset, env->d_counters, env->desc, env->cells};
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

// grows the env's tree slab and refreshes the UCB table for (iters, c)
int prepare(ludax_env* env, int iters, double c, int mask_words, MctsArgs& a) {
    const int cap = iters + 1;
    const size_t node_bytes = sizeof(TNode) * (size_t)cap * (size_t)env->n;
    const size_t mask_bytes = sizeof(uint64_t) * (size_t)mask_words * (size_t)cap * (size_t)env->n;
    const size_t need = node_bytes + mask_bytes;
    if (need > env->tree_bytes) {
        cudaStreamSynchronize(env->stream);
        cudaFree(env->d_tree);
        env->d_tree = nullptr;
        env->tree_bytes = 0;
        if (cudaMalloc(&env->d_tree, need) != cudaSuccess) {
            cudaGetLastError();
            return LUDAX_ERR_NOMEM;
        }
        env->tree_bytes = need;
    }
    if (!env->d_ucb || env->ucb_c != c) {
        std::vector<double> t((size_t)LUDAX_MCTS_MAX_ITERS + 2, 0.0);
        for (int m = 1; m < (int)t.size(); ++m) t[(size_t)m] = c * std::sqrt(std::log((double)m));
        if (!env->d_ucb && cudaMalloc(&env->d_ucb, sizeof(double) * t.size()) != cudaSuccess) {
            cudaGetLastError();
            env->d_ucb = nullptr;
            return LUDAX_ERR_NOMEM;
        }
        if (cudaMemcpyAsync(env->d_ucb, t.data(), sizeof(double) * t.size(), cudaMemcpyHostToDevice, env->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(env->stream) != cudaSuccess)
            return LUDAX_ERR_CUDA;
        env->ucb_len = (int)t.size();
        env->ucb_c = c;
    }
    a.cap_nodes = cap;
    a.T = env->d_ucb;
    a.nodes = (TNode*)env->d_tree;
    a.masks = (uint64_t*)((char*)env->d_tree + node_bytes);
    a.d = dev_of(env);
    a.num_actions = env->num_actions;
    return LUDAX_OK;
}

bool valid_c(double c) { return std::isfinite(c) && c >= 0.0; }

}  // namespace

extern "C" {

int ludax_mcts_search(ludax_env* env, uint64_t seed, int32_t iterations, double c, int32_t* action_dev,
                      uint32_t* visits_dev, uint32_t* wins_dev) {
    if (!env || !action_dev || iterations < 1 || iterations > LUDAX_MCTS_MAX_ITERS || !valid_c(c)) return LUDAX_ERR_ARG;
    if (!aligned(action_dev, 4) || (visits_dev && !aligned(visits_dev, 4)) || (wins_dev && !aligned(wins_dev, 4)))
        return LUDAX_ERR_ALIGN;
    return dispatch_game(env->game, env->rows, env->cols, [&](auto tag) {
        using G = typename decltype(tag)::type;
        MctsArgs a{};
        int st = prepare(env, iterations, c, MaskWords<typename G::Mask>::value, a);
        if (st != LUDAX_OK) return st;
        a.seed_key = splitmix64(seed);
        a.iters_p1 = a.iters_p2 = iterations;
        a.action = action_dev;
        a.visits = visits_dev;
        a.wins = wins_dev;
        const unsigned grid = (unsigned)((env->n + 63) / 64);
        uct_search_kernel<G><<<grid, 64, 0, env->stream>>>(a);
        return cudaGetLastError() == cudaSuccess ? LUDAX_OK : LUDAX_ERR_CUDA;
    });
}

int ludax_mcts_play(ludax_env* env, uint64_t seed, uint32_t flags, int32_t iters_p1, int32_t iters_p2, double c,
                    int8_t* outcome_dev, int16_t* plies_dev, int16_t* agency_dev, int16_t* coverage_dev) {
    if (!env || iters_p1 < 1 || iters_p2 < 1 || iters_p1 > LUDAX_MCTS_MAX_ITERS || iters_p2 > LUDAX_MCTS_MAX_ITERS ||
        !valid_c(c))
        return LUDAX_ERR_ARG;
    if (flags & ~(uint32_t)(LUDAX_ROLLOUT_FROM_START | LUDAX_ROLLOUT_WRITE_BACK)) return LUDAX_ERR_ARG;
    if ((plies_dev && !aligned(plies_dev, 2)) || (agency_dev && !aligned(agency_dev, 2)) ||
        (coverage_dev && !aligned(coverage_dev, 2)))
        return LUDAX_ERR_ALIGN;
    return dispatch_game(env->game, env->rows, env->cols, [&](auto tag) {
        using G = typename decltype(tag)::type;
        MctsArgs a{};
        const int iters = iters_p1 > iters_p2 ? iters_p1 : iters_p2;
        int st = prepare(env, iters, c, MaskWords<typename G::Mask>::value, a);
        if (st != LUDAX_OK) return st;
        a.seed_key = splitmix64(seed);
        a.iters_p1 = iters_p1;
        a.iters_p2 = iters_p2;
        a.from_start = (flags & LUDAX_ROLLOUT_FROM_START) ? 1 : 0;
        a.write_back = (flags & LUDAX_ROLLOUT_WRITE_BACK) ? 1 : 0;
        a.outcome = outcome_dev;
        a.plies = plies_dev;
        a.agency = agency_dev;
        a.coverage = coverage_dev;
        const unsigned grid = (unsigned)((env->n + 63) / 64);
        uct_match_kernel<G><<<grid, 64, 0, env->stream>>>(a);
        return cudaGetLastError() == cudaSuccess ? LUDAX_OK : LUDAX_ERR_CUDA;
    });
}

}  // extern "C"
