// ludax_mcts.cu -- UCT agents (MCTS with the UCB1 rule and a uniform-random
// playout at each new leaf) and whole agent-vs-agent matches, the agents of
// the GAVEL-like evaluation in App. F ("MCTS with UCB1", a number of
// iterations per move, each a traversal, an expansion and a random rollout).
//
// One warp owns one search (or one match, whose searches it runs one after
// the other).  The game state lives in registers and is re-derived along the
// path from the root at every iteration; the tree lives in a per-env slab of
// a scratch buffer: 16-byte nodes {parent, action, first child, next sibling,
// N, W} and one tried-action bitboard per node.  Rewards are integer half
// points (win 2, draw 1, loss 0), so back-propagation is exact and the UCB1
// score W/(2N) + T[N_parent]/sqrt(N) is computed with correctly rounded
// double division and square root; T[m] = c*sqrt(ln m) is tabulated on the
// host.
//
// Warp cooperation without changing the result: while the root still has
// untried actions, an iteration's path is root -> a new child, and which
// child it expands depends only on the iteration's draw and the root's tried
// set, never on earlier playout results.  So up to 32 such iterations form a
// round: every lane replays the round's expansion draws (cheap), takes its
// own iteration's child, plays its playout, and writes its node exactly where
// the sequential search would have (node index, sibling link, N = 1, W); the
// root then adds the round's visits.  Iterations that descend by UCB1 run in
// all lanes on the same data (lane 0 alone writes the tree); their playouts
// share each ply of a move game -- one piece per lane for the move lookup --
// and are computed redundantly otherwise.  Every loop is bounded by the
// iteration count and the game's ply cap.
#include <cmath>
#include <vector>

#include "ludax_internal.cuh"

namespace {
using namespace ludax;

struct TNode {
    int16_t parent, action, first_child, next_sibling;  // action: internal bit (move games: ordinal), -1 = pass
    uint16_t N, W;                                      // N <= 4096 iterations, W <= 2N half points
    int8_t mover;                                       // side that made the move into the node (0 = P1)
    int8_t pad[3];
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

__device__ __forceinline__ TNode make_node(int parent, int action, int first_child, int next_sibling, uint32_t N,
                                           uint32_t W, int mover) {
    return TNode{(int16_t)parent, (int16_t)action, (int16_t)first_child, (int16_t)next_sibling, (uint16_t)N,
                 (uint16_t)W, (int8_t)mover, {0, 0, 0}};
}

__device__ __forceinline__ double ucb1(uint32_t W, uint32_t N, double t) {
    const double n = (double)N;
    return __dadd_rn(__ddiv_rn((double)W, __dmul_rn(2.0, n)), __ddiv_rn(t, __dsqrt_rn(n)));
}

template <class M>
__device__ __forceinline__ M mask_without(M m, int b) {
    if constexpr (MaskWords<M>::value == 1) {
        return m & ~((M)1 << b);
    } else {
        mask_add(m, b);  // make sure the bit is set, then flip it off
        M one{};
        mask_add(one, b);
        return m & ~one;
    }
}

// One sequential iteration (traversal by UCB1, expansion, playout, update)
// with the iteration key ki; count = nodes in use.  All 32 lanes of the warp
// run it on the same data: the traversal and the playout are computed in
// every lane (a move game's playout shares each ply's move lookup across the
// lanes), and lane 0 alone writes the tree.
template <class G>
__device__ void uct_iteration(const G& root, uint64_t ki, const double* __restrict__ T, TNode* nd, uint64_t* mk,
                              int& count, int lane) {
    using M = typename G::Mask;
    constexpr int MW = MaskWords<M>::value;
    G g = root;
    int x = 0;
    while (g.outcome == kOngoing) {
        const M legal = g.legal();
        if (G::kHasPass && !any(legal)) {  // the forced pass is the only action
            if (nd[x].first_child < 0) {
                const int y = count++;
                if (lane == 0) {
                    nd[y] = make_node(x, -1, -1, -1, 0u, 0u, g.side);
                    mask_zero(mk + (size_t)y * MW, MW);
                    nd[x].first_child = (int16_t)y;
                }
                play(g, -1);
                x = y;
                break;
            }
            x = nd[x].first_child;
            play(g, -1);
            continue;
        }
        M tried;
        mask_get(mk + (size_t)x * MW, tried);
        const M untried = legal & ~tried;
        if (any(untried)) {
            const uint32_t k = __umulhi((uint32_t)(splitmix64(~ki) >> 32), popc(untried));
            const int b = select_bit(untried, k);
            mask_add(tried, b);
            const int y = count++;
            if (lane == 0) {
                mask_put(mk + (size_t)x * MW, tried);
                nd[y] = make_node(x, b, -1, nd[x].first_child, 0u, 0u, g.side);
                mask_zero(mk + (size_t)y * MW, MW);
                nd[x].first_child = (int16_t)y;
            }
            play(g, b);
            x = y;
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
    }
    while (g.outcome == kOngoing) random_ply_warp(g, ki, lane);
    if (lane == 0) {  // the new node's links were written by this lane
        for (int y = x; y > 0; y = nd[y].parent) {
            nd[y].N = (uint16_t)(nd[y].N + 1u);
            nd[y].W = (uint16_t)(nd[y].W + half_points(g.outcome, nd[y].mover));
        }
        nd[0].N = (uint16_t)(nd[0].N + 1u);
    }
}

// the move: most visits, then largest W, then smallest action
__device__ __forceinline__ int uct_best(const TNode* nd) {
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

// One search from `root` by a whole warp (all 32 lanes call it with the same
// arguments); returns the chosen action (internal bit, -1 = pass) in every
// lane.  nd / mk: the warp's node slab and tried masks (iters + 1 nodes).
template <class G>
__device__ int uct_search_warp(const G& root, uint64_t key, int iters, const double* __restrict__ T, TNode* nd,
                               uint64_t* mk, int lane) {
    using M = typename G::Mask;
    constexpr int MW = MaskWords<M>::value;
    if (lane == 0) {
        nd[0] = make_node(-1, -1, -1, -1, 0u, 0u, 0);
        mask_zero(mk, MW);
    }
    __syncwarp();
    const M legal = root.legal();
    const bool forced_pass = G::kHasPass && !any(legal);
    int count = 1, i = 0;
    while (i < iters) {
        M tried;
        mask_get(mk, tried);
        const M untried = legal & ~tried;
        if (!forced_pass && any(untried)) {
            // a round of root expansions, one iteration per lane
            int R = iters - i < 32 ? iters - i : 32;
            const int nu = (int)popc(untried);
            R = nu < R ? nu : R;
            M u = untried;
            int mine = -1;
            for (int j = 0; j < R; ++j) {
                const uint64_t kj = splitmix64(key ^ (uint64_t)(i + j));
                const int b = select_bit(u, __umulhi((uint32_t)(splitmix64(~kj) >> 32), popc(u)));
                if (j == lane) mine = b;
                u = mask_without(u, b);
            }
            const int16_t head = nd[0].first_child;
            __syncwarp();
            if (lane < R) {
                G g = root;
                play(g, mine);
                const uint64_t ki = splitmix64(key ^ (uint64_t)(i + lane));
                while (g.outcome == kOngoing) random_ply(g, ki);
                const int y = count + lane;
                nd[y] = make_node(0, mine, -1, lane == 0 ? head : y - 1, 1u, half_points(g.outcome, root.side),
                                  root.side);
                mask_zero(mk + (size_t)y * MW, MW);
            }
            if (lane == 0) {
                nd[0].first_child = (int16_t)(count + R - 1);
                nd[0].N = (uint16_t)(nd[0].N + R);
                mask_put(mk, tried | (untried & ~u));
            }
            count += R;
            i += R;
        } else {
            uct_iteration(root, splitmix64(key ^ (uint64_t)i), T, nd, mk, count, lane);
            ++i;
        }
        __syncwarp();
    }
    int best = 0;
    if (lane == 0) best = uct_best(nd);
    return __shfl_sync(0xffffffffu, best, 0);
}

__device__ __forceinline__ uint64_t search_key(uint64_t seed_key, int64_t match, int ply) {
    return splitmix64(env_key(seed_key, (uint64_t)match) ^ ((uint64_t)(ply + 1) << 32));
}

struct MctsArgs {
    EnvDev d;
    uint64_t seed_key;  // splitmix64(seed)
    int iters_p1, iters_p2, cap_nodes, num_actions, slab_words;
    const double* T;
    TNode* nodes;
    uint64_t* masks;
    // search mode
    int32_t* action;
    uint32_t* visits;
    uint32_t* wins;
    // match mode
    int from_start, write_back;
    const int32_t* desc;   // mixed matches: per-env descriptor
    const int32_t* iters;  // mixed matches: per-env [P1, P2] iterations
    int8_t* outcome;
    int16_t* plies;
    int16_t* agency;
    int16_t* coverage;
};

constexpr int kWarpsPerBlock = 2;

// The match of env e played by one warp (from the start position or from g).
template <class G>
__device__ void play_match(G& g, const MctsArgs& a, int64_t e, int64_t match, int iters_p1, int iters_p2, int lane) {
    constexpr int MW = MaskWords<typename G::Mask>::value;
    TNode* nd = a.nodes + (size_t)e * a.cap_nodes;
    uint64_t* mk = a.masks + (size_t)e * a.cap_nodes * a.slab_words;
    auto ever = occupied_of(g);
    int turns = 0;
    (void)MW;
    while (g.outcome == kOngoing) {
        const typename G::Mask legal = g.legal();
        int b = -1;
        if (!(G::kHasPass && !any(legal))) {
            if (popc(legal) > 1) {
                ++turns;
                b = uct_search_warp(g, search_key(a.seed_key, match, g.ply), g.side == 0 ? iters_p1 : iters_p2, a.T,
                                    nd, mk, lane);
            } else {
                b = select_bit(legal, 0u);
            }
        }
        play(g, b);
        ever = ever | occupied_of(g);
    }
    if (lane == 0) {
        if (a.outcome) a.outcome[e] = (int8_t)g.outcome;
        if (a.plies) a.plies[e] = (int16_t)g.ply;
        if (a.agency) a.agency[e] = (int16_t)turns;
        if (a.coverage) a.coverage[e] = (int16_t)popc(ever);
    }
}

__device__ __forceinline__ int64_t warp_env() {
    return (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
}

template <class G>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) uct_search_kernel(MctsArgs a) {
    const int64_t e = warp_env();
    const int lane = threadIdx.x & 31;
    if (e >= a.d.n) return;  // whole warps leave together
    TNode* nd = a.nodes + (size_t)e * a.cap_nodes;
    uint64_t* mk = a.masks + (size_t)e * a.cap_nodes * a.slab_words;
    G g;
    set_table(g, nullptr);
    load_state(g, a.d, e);
    int act = -1;
    if (g.outcome == kOngoing) {
        const int b = uct_search_warp(g, search_key(a.seed_key, a.d.env_offset + e, g.ply), a.iters_p1, a.T, nd, mk,
                                      lane);
        act = b < 0 ? G::kCells : g.canon_of(b);
    }
    if (lane == 0) a.action[e] = act;
    if (a.visits || a.wins) {
        const size_t row = (size_t)e * a.num_actions;
        for (int j = lane; j < a.num_actions; j += 32) {
            if (a.visits) a.visits[row + j] = 0u;
            if (a.wins) a.wins[row + j] = 0u;
        }
        __syncwarp();
        if (lane == 0 && act >= 0) {
            for (int y = nd[0].first_child; y >= 0; y = nd[y].next_sibling) {
                const int j = nd[y].action < 0 ? G::kCells : g.canon_of(nd[y].action);
                if (a.visits) a.visits[row + j] = nd[y].N;
                if (a.wins) a.wins[row + j] = nd[y].W;
            }
        }
    }
}

template <class G>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) uct_match_kernel(MctsArgs a) {
    const int64_t e = warp_env();
    const int lane = threadIdx.x & 31;
    if (e >= a.d.n) return;
    G g;
    set_table(g, nullptr);
    if (a.from_start) {
        configure(g, a.d.desc);
        g.reset();
    } else {
        load_state(g, a.d, e);
    }
    play_match(g, a, e, a.d.env_offset + e, a.iters_p1, a.iters_p2, lane);
    if (a.write_back && lane == 0) store_state(g, a.d, e);
}

// Matches of any mix of games: the warp of env e reads its descriptor and
// runs that game's code (the game is uniform across the warp).
template <class G>
__device__ __forceinline__ void mixed_match(const MctsArgs& a, int64_t e, int lane) {
    G g;
    set_table(g, nullptr);
    configure(g, a.desc[e]);
    g.reset();
    play_match(g, a, e, a.d.env_offset + e, a.iters[2 * e], a.iters[2 * e + 1], lane);
}

__global__ void __launch_bounds__(32 * kWarpsPerBlock) uct_match_mixed_kernel(MctsArgs a) {
    const int64_t e = warp_env();
    const int lane = threadIdx.x & 31;
    if (e >= a.d.n) return;
    switch (desc_bucket(a.desc[e])) {
    case 0: mixed_match<TTT>(a, e, lane); break;
    case 1: mixed_match<C4>(a, e, lane); break;
    case 2: mixed_match<Othello>(a, e, lane); break;
    case 3: mixed_match<Hex<2>>(a, e, lane); break;
    case 4: mixed_match<Hex<3>>(a, e, lane); break;
    case 5: mixed_match<Hex<4>>(a, e, lane); break;
    case 6: mixed_match<Hex<5>>(a, e, lane); break;
    case 7: mixed_match<Hex<6>>(a, e, lane); break;
    case 8: mixed_match<Hex<7>>(a, e, lane); break;
    case 9: mixed_match<Hex<8>>(a, e, lane); break;
    case 10: mixed_match<Hex<9>>(a, e, lane); break;
    case 11: mixed_match<Hex<10>>(a, e, lane); break;
    case 12: mixed_match<Hex<11>>(a, e, lane); break;
    case 13: mixed_match<Gomoku>(a, e, lane); break;
    case 14: mixed_match<Pente>(a, e, lane); break;
    case 15: mixed_match<Yavalath>(a, e, lane); break;
    case 16: mixed_match<LineGame>(a, e, lane); break;
    case 17: mixed_match<WolfSheep>(a, e, lane); break;
    case 18: mixed_match<Draughts>(a, e, lane); break;
    case 19: mixed_match<HasamiShogi>(a, e, lane); break;
    default: break;  // validated on the host
    }
}

EnvDev dev_of(const ludax_env* env) {
    return EnvDev{env->d_planes, env->d_meta, env->n, env->env_offset, env->d_counters, env->desc, env->cells};
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

unsigned warp_grid(int64_t n) { return (unsigned)((n + kWarpsPerBlock - 1) / kWarpsPerBlock); }

bool valid_c(double c) { return std::isfinite(c) && c >= 0.0; }

std::vector<double> ucb_table(double c) {
    std::vector<double> t((size_t)LUDAX_MCTS_MAX_ITERS + 2, 0.0);
    for (int m = 1; m < (int)t.size(); ++m) t[(size_t)m] = c * std::sqrt(std::log((double)m));
    return t;
}

// grows the env's tree slab and refreshes its UCB table for (iters, c)
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
        const std::vector<double> t = ucb_table(c);
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
    a.slab_words = mask_words;
    a.T = env->d_ucb;
    a.nodes = (TNode*)env->d_tree;
    a.masks = (uint64_t*)((char*)env->d_tree + node_bytes);
    a.d = dev_of(env);
    a.num_actions = env->num_actions;
    return LUDAX_OK;
}

}  // namespace

extern "C" {

int ludax_mcts_reserve(ludax_env* env, int32_t iterations, double c) {
    if (!env || iterations < 1 || iterations > LUDAX_MCTS_MAX_ITERS || !valid_c(c)) return LUDAX_ERR_ARG;
    return dispatch_game(env->game, env->rows, env->cols, [&](auto tag) {
        using G = typename decltype(tag)::type;
        MctsArgs a{};
        return prepare(env, iterations, c, MaskWords<typename G::Mask>::value, a);
    });
}

int ludax_mcts_search(ludax_env* env, uint64_t seed, int32_t iterations, double c, int32_t* action_dev,
                      uint32_t* visits_dev, uint32_t* wins_dev) {
    ludax::ApiRange api_range("ludax_mcts_search");
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
        uct_search_kernel<G><<<warp_grid(env->n), 32 * kWarpsPerBlock, 0, env->stream>>>(a);
        return cudaGetLastError() == cudaSuccess ? LUDAX_OK : LUDAX_ERR_CUDA;
    });
}

int ludax_mcts_play(ludax_env* env, uint64_t seed, uint32_t flags, int32_t iters_p1, int32_t iters_p2, double c,
                    int8_t* outcome_dev, int16_t* plies_dev, int16_t* agency_dev, int16_t* coverage_dev) {
    ludax::ApiRange api_range("ludax_mcts_play");
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
        uct_match_kernel<G><<<warp_grid(env->n), 32 * kWarpsPerBlock, 0, env->stream>>>(a);
        return cudaGetLastError() == cudaSuccess ? LUDAX_OK : LUDAX_ERR_CUDA;
    });
}

int ludax_mcts_play_mixed(const int32_t* desc_host, const int32_t* iters_host, int64_t n, int64_t env_offset,
                          uint64_t seed, double c, int8_t* outcome_dev, int16_t* plies_dev, int16_t* agency_dev,
                          int16_t* coverage_dev, void* stream, int64_t* bad_index) {
    ludax::ApiRange api_range("ludax_mcts_play_mixed");
    if (bad_index) *bad_index = -1;
    if (!desc_host || !iters_host || n < 1 || n > 0x7FFFFFFFll || env_offset < 0 || !valid_c(c)) return LUDAX_ERR_ARG;
    if ((plies_dev && !aligned(plies_dev, 2)) || (agency_dev && !aligned(agency_dev, 2)) ||
        (coverage_dev && !aligned(coverage_dev, 2)))
        return LUDAX_ERR_ALIGN;
    int max_iters = 1;
    for (int64_t e = 0; e < n; ++e) {
        const int b = desc_bucket(desc_host[e]);
        const int i1 = iters_host[2 * e], i2 = iters_host[2 * e + 1];
        if (b < 0 || i1 < 1 || i2 < 1 || i1 > LUDAX_MCTS_MAX_ITERS || i2 > LUDAX_MCTS_MAX_ITERS) {
            if (bad_index) *bad_index = e;
            return b == -1 ? LUDAX_ERR_GAME : (b == -2 ? LUDAX_ERR_SIZE : LUDAX_ERR_ARG);
        }
        max_iters = i1 > max_iters ? i1 : max_iters;
        max_iters = i2 > max_iters ? i2 : max_iters;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int cap = max_iters + 1, words = 6;  // the widest legal mask (Pente)
    const size_t node_bytes = sizeof(TNode) * (size_t)cap * (size_t)n;
    const size_t mask_bytes = sizeof(uint64_t) * words * (size_t)cap * (size_t)n;
    const std::vector<double> t = ucb_table(c);
    const size_t table_bytes = sizeof(double) * t.size();
    const size_t in_bytes = sizeof(int32_t) * 3 * (size_t)n;
    char* scratch = nullptr;
    if (cudaMallocAsync((void**)&scratch, node_bytes + mask_bytes + table_bytes + in_bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return LUDAX_ERR_NOMEM;
    }
    MctsArgs a{};
    a.nodes = (TNode*)scratch;
    a.masks = (uint64_t*)(scratch + node_bytes);
    double* d_table = (double*)(scratch + node_bytes + mask_bytes);
    int32_t* d_in = (int32_t*)(scratch + node_bytes + mask_bytes + table_bytes);
    int st = LUDAX_OK;
    // pageable host sources: the copies complete before cudaMemcpyAsync returns
    if (cudaMemcpyAsync(d_table, t.data(), table_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(d_in, desc_host, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(d_in + n, iters_host, sizeof(int32_t) * 2 * (size_t)n, cudaMemcpyHostToDevice, s) !=
            cudaSuccess) {
        st = LUDAX_ERR_CUDA;
    } else {
        a.d = EnvDev{nullptr, nullptr, n, env_offset, nullptr, 0, 0};
        a.seed_key = splitmix64(seed);
        a.cap_nodes = cap;
        a.slab_words = words;
        a.T = d_table;
        a.desc = d_in;
        a.iters = d_in + n;
        a.outcome = outcome_dev;
        a.plies = plies_dev;
        a.agency = agency_dev;
        a.coverage = coverage_dev;
        uct_match_mixed_kernel<<<warp_grid(n), 32 * kWarpsPerBlock, 0, s>>>(a);
        if (cudaGetLastError() != cudaSuccess) st = LUDAX_ERR_CUDA;
    }
    cudaFreeAsync(scratch, s);
    return st;
}

}  // extern "C"
