// ludax_umma.cu -- dense BF16 layer on the 5th-generation tensor cores:
//   out[m][n] = bf16( relu( sum_k A[m][k] * B[n][k] + bias[n] ) )
// A [M][K] and B [N][K] are row-major (K contiguous) BF16, FP32 accumulation.
//
// Persistent, warp-specialised kernel: one CTA per SM walks 128 x 256 output
// tiles (tile t covers rows 128*(t / (N/256)) and columns 256*(t % (N/256))).
//   warp 0    : TMA producer -- streams 128x64 (A) and 256x64 (B) K-slices
//               (cp.async.bulk.tensor, 128-byte swizzle) into a 4-stage
//               shared-memory ring guarded by full/empty mbarriers;
//   warp 1    : MMA issuer -- one thread issues tcgen05.mma (kind::f16,
//               M=128, N=256, K=16) into one of two 256-column FP32
//               accumulators in TMEM, frees ring stages with tcgen05.commit
//               and signals the finished accumulator;
//   warps 2-5 : epilogue -- drain the finished accumulator with tcgen05.ld
//               (each warp its quarter of the 128 TMEM lanes = rows; the load
//               of the next 32 columns is in flight while the current ones
//               are converted), add the bias (staged in shared memory),
//               ReLU, round to BF16 into a 32 x 64 shared-memory box in the
//               128-byte-swizzle layout (conflict-free), and store each box
//               with one bulk tensor store (cp.async.bulk.tensor); then hand
//               the accumulator back, so the epilogue of tile i overlaps the
//               MMAs of tile i+1.
// Every mbarrier wait is bounded (about a second of clock); on expiry the
// kernel records an error in a device word and stops issuing work, so a
// fault in the pipeline surfaces as a status instead of a hang.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>
#include <set>
#include <utility>

#include "ludax_internal.cuh"

namespace {

constexpr int TM = 128, TN = 256, TK = 64, UMMA_THREADS = 192;
constexpr int A_TILE = TM * TK * 2, B_TILE = TN * TK * 2, STAGE = A_TILE + B_TILE;
constexpr int TMEM_COLS = 2 * TN;  // two accumulators
constexpr int MAX_N = 1024;        // the bias row is staged in shared memory
constexpr int OUT_BOX = 64;        // output columns per TMA store box (128 bytes of BF16)
constexpr int BOX_BYTES = 32 * OUT_BOX * 2;  // one 32-row x 64-column BF16 box, 128-byte swizzle
constexpr int DENSE_STAGES = 4;              // dense layer: ring depth; one staging box per epilogue warp
constexpr int RING = DENSE_STAGES * STAGE;
constexpr size_t UMMA_SMEM = 1024 /* alignment */ + (size_t)RING + 4 * BOX_BYTES + 256 /* barriers */ +
                             2 * sizeof(float) * MAX_N /* bias, head weights */;
constexpr long long kWaitLimit = 2000000000ll;  // clock cycles (~1 s at 2 GHz)

static __device__ int g_umma_error;  // nonzero after a wait expired

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(saddr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for the phase with the given parity to complete; false after kWaitLimit cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitLimit) return false;
    return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];\n" ::
            "r"(saddr(dst)),
        "l"(map), "r"(saddr(bar)), "r"(c0), "r"(c1)
        : "memory");
}

// The same load with an L2 eviction policy (createpolicy) for the lines it reads.
__device__ __forceinline__ void tma_load_2d_hint(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                                 uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%3, "
        "%4}], [%2], %5;\n" ::"r"(saddr(dst)),
        "l"(map), "r"(saddr(bar)), "r"(c0), "r"(c1), "l"(policy)
        : "memory");
}
// a policy under which L2 gives up the lines first (data read for the last time)
__device__ __forceinline__ uint64_t l2_last_use_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
    return p;
}
__device__ __forceinline__ void tma_load_2d_pol(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                                uint64_t policy) {
    if (policy) tma_load_2d_hint(dst, map, bar, c0, c1, policy);
    else tma_load_2d(dst, map, bar, c0, c1);
}

// bulk tensor store of a shared-memory box to global memory (bulk async-group)
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int c0, int c1) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];\n" ::"l"(map),
                 "r"(saddr(src)), "r"(c0), "r"(c1)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}
// the shared-memory sources of this thread's bulk stores (all, or all but the most recent) may be overwritten
__device__ __forceinline__ void tma_store_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
__device__ __forceinline__ void tma_store_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;\n" ::: "memory"); }
__device__ __forceinline__ void tma_store_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// Shared-memory matrix descriptor for a K-major operand tile written by TMA
// with 128-byte swizzle: rows of 128 bytes, 8-row atoms 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)1 << 16;                            // leading byte offset (unused with this swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;                  // stride byte offset: next 8-row atom
    d |= (uint64_t)1 << 46;                            // descriptor version
    d |= (uint64_t)2 << 61;                            // 128-byte swizzle
    return d;
}

// Instruction descriptor: D FP32, A and B BF16, both K-major, N = TN, M = TM.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(saddr(bar))
                 : "memory");
}

// 32 columns of this warp's 32 TMEM lanes into r (asynchronous: tmem_wait_ld)
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
// waits for the outstanding TMEM loads; r (the registers they fill) are
// read-write operands, so no use of them is moved before the wait
__device__ __forceinline__ void tmem_wait_ld(uint32_t* r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

// Drains NCH 32-column chunks, from chunk c0 on, of one accumulator (this
// warp's 32 TMEM lanes = rows): the load of the next chunk is in flight
// while the current one is converted.  For each chunk c, fn(c, v) gets this
// lane's 32 values of relu(acc + bias) as 16 BF16 pairs.
template <int NCH, class F>
__device__ __forceinline__ void drain_accumulator(uint32_t base, int c0, const float* bias_n0, F&& fn) {
    uint32_t r[2][32];
    tmem_ld32_async(base + (uint32_t)(c0 * 32), r[0]);
    tmem_wait_ld(r[0]);
#pragma unroll
    for (int i = 0; i < NCH; ++i) {
        const int c = c0 + i;
        if (i + 1 < NCH) tmem_ld32_async(base + (uint32_t)((c + 1) * 32), r[(i + 1) & 1]);
        const uint32_t* x = r[i & 1];
        const float4* bb = reinterpret_cast<const float4*>(bias_n0 + c * 32);
        __align__(16) __nv_bfloat162 v[16];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float4 b4 = bb[j];
            v[2 * j] = __floats2bfloat162_rn(fmaxf(__uint_as_float(x[4 * j]) + b4.x, 0.f),
                                             fmaxf(__uint_as_float(x[4 * j + 1]) + b4.y, 0.f));
            v[2 * j + 1] = __floats2bfloat162_rn(fmaxf(__uint_as_float(x[4 * j + 2]) + b4.z, 0.f),
                                                 fmaxf(__uint_as_float(x[4 * j + 3]) + b4.w, 0.f));
        }
        fn(c, v);
        if (i + 1 < NCH) tmem_wait_ld(r[(i + 1) & 1]);
    }
}

// <v, w[0..31]> over one chunk of BF16 activations (four partial sums, so
// the multiply-adds are not one dependent chain)
__device__ __forceinline__ float dot_chunk(const __nv_bfloat162* v, const float* w) {
    const float4* ww = reinterpret_cast<const float4*>(w);
    float z0 = 0.f, z1 = 0.f, z2 = 0.f, z3 = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float4 w4 = ww[j];
        const float2 f0 = __bfloat1622float2(v[2 * j]), f1 = __bfloat1622float2(v[2 * j + 1]);
        z0 = fmaf(f0.x, w4.x, z0);
        z1 = fmaf(f0.y, w4.y, z1);
        z2 = fmaf(f1.x, w4.z, z2);
        z3 = fmaf(f1.y, w4.w, z3);
    }
    return (z0 + z1) + (z2 + z3);
}

// One 32-column chunk of BF16 values into this lane's row of a 32 x 64
// staging box (128-byte swizzle), and the box to global memory by TMA once
// both of its chunks are in.  With BOXES = 2 the warp's two boxes alternate
// (box of chunk c = (c / 2) % 2), so a box fills while the store of the
// other is still reading it out: before a box is refilled, at most one store
// (the other box's) may be pending.
template <int BOXES>
__device__ __forceinline__ void stage_chunk(int c, const __nv_bfloat162* v, uint8_t* staging_warp, int lane,
                                            const CUtensorMap* map, int col_base, int row0) {
    uint8_t* box = staging_warp + (BOXES == 2 ? ((c >> 1) & 1) * BOX_BYTES : 0);
    uint8_t* myrow = box + lane * (OUT_BOX * 2);
    const int half = c & 1;
    if (half == 0) {
        if (lane == 0) {
            if (BOXES == 2) tma_store_wait_read1();
            else tma_store_wait_read0();
        }
        __syncwarp();
    }
    const uint4* src = reinterpret_cast<const uint4*>(v);
#pragma unroll
    for (int k = 0; k < 4; ++k) {  // 16-byte chunk 4*half+k of the row, swizzled with the row
        const int chunk = (4 * half + k) ^ (lane & 7);
        *reinterpret_cast<uint4*>(myrow + chunk * 16) = src[k];
    }
    if (half == 1) {  // box complete: hand it to the TMA engine
        fence_async_shared();
        __syncwarp();
        if (lane == 0) tma_store_2d(map, box, col_base + (c - 1) * 32, row0);
    }
}

// Bit k of the result: value k of the 32 BF16 values v (non-negative, as
// ReLU leaves them) is non-zero.  Per 32-bit word, adding 0x7FFF to each
// half's magnitude carries into the half's top bit exactly when the half is
// non-zero (a -0 from the ReLU counts as zero, as in a "> 0" test).
__device__ __forceinline__ uint32_t nonzero_bits(const __nv_bfloat162* v) {
    const uint32_t* w = reinterpret_cast<const uint32_t*>(v);
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const uint32_t t = ((w[k] & 0x7FFF7FFFu) + 0x7FFF7FFFu) & 0x80008000u;
        m |= ((t >> 15) & 1u) << (2 * k) | (t >> 31) << (2 * k + 1);
    }
    return m;
}

__global__ void __launch_bounds__(UMMA_THREADS, 1)
    umma_dense_relu_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                           const __grid_constant__ CUtensorMap tmOut, int M, int N, int K,
                           const float* __restrict__ bias, const __nv_bfloat16* __restrict__ w3,
                           float* __restrict__ zpart, int store) {
    ludax::pdl_wait();
    extern __shared__ __align__(16) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t* staging = smem + RING;  // 1024-byte aligned: the 128-byte swizzle pattern repeats every 1024 bytes
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + RING + 4 * BOX_BYTES);
    uint64_t* empty = full + DENSE_STAGES;
    uint64_t* acc_full = empty + DENSE_STAGES;  // [2] MMA -> epilogue
    uint64_t* acc_empty = acc_full + 2;    // [2] epilogue -> MMA
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
    float* sbias = reinterpret_cast<float*>(smem + RING + 4 * BOX_BYTES + 256);
    float* sw3 = sbias + MAX_N;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ktiles = K / TK, ntn = N / TN, ntiles = (M / TM) * ntn;
    const bool head = w3 != nullptr;  // fused head: per-row dot products with w3 (and the rows stored if store)
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        sbias[i] = bias[i];
        sw3[i] = head ? __bfloat162float(w3[i]) : 0.f;
    }

    if (threadIdx.x == 0) {
        for (int s = 0; s < DENSE_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&acc_full[a], 1);
            mbar_init(&acc_empty[a], 128);  // every epilogue thread arrives
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(saddr(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (warp == 0) {
        if (lane == 0) {  // TMA producer
            int it = 0;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                const int m0 = (t / ntn) * TM, n0 = (t % ntn) * TN;
                for (int kt = 0; kt < ktiles && ok; ++kt, ++it) {
                    const int s = it % DENSE_STAGES;
                    if (it >= DENSE_STAGES) ok = mbar_wait(&empty[s], (uint32_t)(((it / DENSE_STAGES) & 1) ^ 1));
                    if (!ok) break;
                    uint8_t* st = smem + s * STAGE;
                    mbar_expect_tx(&full[s], STAGE);
                    tma_load_2d(st, &tmA, &full[s], kt * TK, m0);
                    tma_load_2d(st + A_TILE, &tmB, &full[s], kt * TK, n0);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            int it = 0, local = 0;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++local) {
                const int a = local & 1;
                if (local >= 2) ok = mbar_wait(&acc_empty[a], (uint32_t)(((local >> 1) & 1) ^ 1));
                if (!ok) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(a * TN);
                for (int kt = 0; kt < ktiles && ok; ++kt, ++it) {
                    const int s = it % DENSE_STAGES;
                    ok = mbar_wait(&full[s], (uint32_t)((it / DENSE_STAGES) & 1));
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t sa = saddr(smem + s * STAGE);
                    const uint64_t ad = sw128_desc(sa), bd = sw128_desc(sa + A_TILE);
#pragma unroll
                    for (int kk = 0; kk < TK / 16; ++kk)  // 16 elements = 32 bytes = 2 descriptor units
                        umma_bf16(d, ad + 2 * kk, bd + 2 * kk, (kt | kk) != 0);
                    umma_commit(&empty[s]);
                }
                umma_commit(&acc_full[a]);
            }
        }
    } else {  // epilogue warps 2..5: TMEM lane quarter = warp % 4
        const int q = warp & 3;
        int local = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++local) {
            const int a = local & 1;
            if (ok) ok = mbar_wait(&acc_full[a], (uint32_t)((local >> 1) & 1));
            ok = __all_sync(0xFFFFFFFFu, ok);  // tcgen05.ld is warp-collective
            if (!ok) break;
            tc_fence_after();
            const int row0 = (t / ntn) * TM + q * 32, n0 = (t % ntn) * TN;
            uint8_t* box = staging + q * BOX_BYTES;
            const uint32_t base = tmem + (uint32_t)(a * TN) + ((uint32_t)(q * 32) << 16);
            float z = 0.f;  // fused head: this row's dot product over the tile's columns
            drain_accumulator<TN / 32>(base, 0, sbias + n0, [&](int c, const __nv_bfloat162* v) {
                if (head) z += dot_chunk(v, sw3 + n0 + c * 32);  // the BF16 activations times w3
                if (store) stage_chunk<1>(c, v, box, lane, &tmOut, n0, row0);
            });
            if (head) zpart[(size_t)(row0 + lane) * ntn + (t % ntn)] = z;
            tc_fence_before();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(saddr(&acc_empty[a])) : "memory");
        }
    }
    if (!ok) atomicOr(&g_umma_error, 1);
    if (warp >= 2 && lane == 0) tma_store_wait_all();  // the epilogue's bulk stores have landed
    tc_fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS));
}

// --------------------------------------------- fused inference MLP --
// Both hidden layers (N = 512) and the head for 128-row blocks in one
// persistent launch.  For block i of this CTA, layer 1 (two 256-column
// halves, K1 input columns) writes its BF16 rows to this CTA's scratch slot
// i % 2 in global memory -- reused block after block, so it stays in L2 and
// never reaches HBM -- and one block later, while the stores drain behind the
// next block's layer 1, layer 2 reads them back through TMA and the head
// takes each row's dot product with w3.  Jobs in order: L1(0), L1(1), L2(0),
// L1(2), L2(1), ..., L2(nb - 1); each job is one 128 x 256 tile through a
// 3-stage ring and two TMEM accumulators.  Draining an accumulator is the
// slow part of a job (a 128 x 256 drain took ~2.4 us with four epilogue
// warps, against ~1.1 us of MMAs for a K = 192 layer-1 tile), so eight
// epilogue warps split it: warps w and w + 4 share TMEM lane quarter w % 4
// and take one 128-column half each; a row's head therefore has four
// partials, zpart[m * 4 + 2 * (column half of the tile) + (half of it)].
// Training form (train != 0): layer 1's rows go to the block's own rows of
// H1 (tmHst / tmHld over H1) instead of a scratch slot -- read back one block
// later while still in L2, and kept for the backward pass -- and layer 2's
// epilogue stores its rows to H2 (tmH2) besides the head's partials.
constexpr int MLP_N = 512;
constexpr int MLP_STAGES = 3, MLP_EPI_WARPS = 8, MLP_THREADS = 32 * (2 + MLP_EPI_WARPS);
constexpr int MLP_STAGING = 2 * BOX_BYTES;  // per epilogue warp: two alternating boxes
constexpr size_t MLP_SMEM = 1024 /* alignment */ + (size_t)MLP_STAGES * STAGE + MLP_EPI_WARPS * MLP_STAGING +
                            256 /* barriers */ + 3 * sizeof(float) * MLP_N /* b1, b2, w3 */;

struct MlpJob {
    int phase, blk, h;  // layer 1 or 2, this CTA's block index, column half
};
__device__ __forceinline__ MlpJob mlp_job(int j, int nb) {
    const int p = j >> 1;
    MlpJob r;
    r.h = j & 1;
    if (p == 0) {
        r.phase = 1, r.blk = 0;
    } else if (p == 2 * nb - 1) {
        r.phase = 2, r.blk = nb - 1;
    } else if (p & 1) {
        r.phase = 1, r.blk = (p + 1) >> 1;
    } else {
        r.phase = 2, r.blk = (p >> 1) - 1;
    }
    return r;
}
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;\n" ::: "memory"); }

__global__ void __launch_bounds__(MLP_THREADS, 1)
    umma_mlp_head_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW1,
                         const __grid_constant__ CUtensorMap tmHst, const __grid_constant__ CUtensorMap tmHld,
                         const __grid_constant__ CUtensorMap tmW2, const __grid_constant__ CUtensorMap tmH2, int M,
                         int K1, const float* __restrict__ b1, const float* __restrict__ b2,
                         const __nv_bfloat16* __restrict__ w3, float* __restrict__ zpart, int train,
                         uint32_t* __restrict__ h1bits) {
    ludax::pdl_wait();
    extern __shared__ __align__(16) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t* staging = smem + MLP_STAGES * STAGE;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + MLP_STAGES * STAGE + MLP_EPI_WARPS * MLP_STAGING);
    uint64_t* empty = full + MLP_STAGES;
    uint64_t* acc_full = empty + MLP_STAGES;  // [2] MMA -> epilogue
    uint64_t* acc_empty = acc_full + 2;    // [2] epilogue -> MMA
    uint64_t* h1_ready = acc_empty + 2;    // [2] epilogue -> producer: a scratch slot's rows are stored
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(h1_ready + 2);
    float* sb1 = reinterpret_cast<float*>(smem + MLP_STAGES * STAGE + MLP_EPI_WARPS * MLP_STAGING + 256);
    float* sb2 = sb1 + MLP_N;
    float* sw3 = sb2 + MLP_N;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nblk = M / TM;
    const int nb = (int)blockIdx.x < nblk ? (nblk - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int njobs = 4 * nb, k1t = K1 / TK, k2t = MLP_N / TK;
    for (int i = threadIdx.x; i < MLP_N; i += blockDim.x) {
        sb1[i] = b1[i];
        sb2[i] = b2[i];
        sw3[i] = __bfloat162float(w3[i]);
    }
    if (threadIdx.x == 0) {
        for (int st = 0; st < MLP_STAGES; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&acc_full[a], 1);
            mbar_init(&acc_empty[a], 32 * MLP_EPI_WARPS);  // every epilogue thread arrives
            mbar_init(&h1_ready[a], MLP_EPI_WARPS);         // lane 0 of each epilogue warp, once its stores are complete
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(saddr(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int scratch0 = (int)blockIdx.x * 2 * TM;  // this CTA's two slots of 128 rows
    bool ok = true;

    if (warp == 0) {
        if (lane == 0) {  // TMA producer
            const uint64_t x_policy = l2_last_use_policy();
            int it = 0;
            for (int j = 0; j < njobs && ok; ++j) {
                const MlpJob jb = mlp_job(j, nb);
                const int gblk = (int)blockIdx.x + jb.blk * (int)gridDim.x;
                if (jb.phase == 2 && jb.h == 0) {  // layer 1's rows of this block must be in global memory
                    ok = mbar_wait(&h1_ready[jb.blk & 1], (uint32_t)((jb.blk >> 1) & 1));
                    if (!ok) break;
                    fence_proxy_async_global();
                }
                const int kt_n = jb.phase == 1 ? k1t : k2t;
                for (int kt = 0; kt < kt_n && ok; ++kt, ++it) {
                    const int st = it % MLP_STAGES;
                    if (it >= MLP_STAGES) ok = mbar_wait(&empty[st], (uint32_t)(((it / MLP_STAGES) & 1) ^ 1));
                    if (!ok) break;
                    uint8_t* dst = smem + st * STAGE;
                    mbar_expect_tx(&full[st], STAGE);
                    if (jb.phase == 1) {
                        // inference reads its input rows once; training's are read again by dW1
                        tma_load_2d_pol(dst, &tmX, &full[st], kt * TK, gblk * TM, train ? 0ull : x_policy);
                        tma_load_2d(dst + A_TILE, &tmW1, &full[st], kt * TK, jb.h * TN);
                    } else {
                        tma_load_2d(dst, &tmHld, &full[st], kt * TK, train ? gblk * TM : scratch0 + (jb.blk & 1) * TM);
                        tma_load_2d(dst + A_TILE, &tmW2, &full[st], kt * TK, jb.h * TN);
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            int it = 0;
            for (int j = 0; j < njobs && ok; ++j) {
                const int a = j & 1;
                if (j >= 2) ok = mbar_wait(&acc_empty[a], (uint32_t)(((j >> 1) & 1) ^ 1));
                if (!ok) break;
                tc_fence_after();
                const int kt_n = mlp_job(j, nb).phase == 1 ? k1t : k2t;
                const uint32_t d = tmem + (uint32_t)(a * TN);
                for (int kt = 0; kt < kt_n && ok; ++kt, ++it) {
                    const int st = it % MLP_STAGES;
                    ok = mbar_wait(&full[st], (uint32_t)((it / MLP_STAGES) & 1));
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t sa = saddr(smem + st * STAGE);
                    const uint64_t ad = sw128_desc(sa), bd = sw128_desc(sa + A_TILE);
#pragma unroll
                    for (int kk = 0; kk < TK / 16; ++kk) umma_bf16(d, ad + 2 * kk, bd + 2 * kk, (kt | kk) != 0);
                    umma_commit(&empty[st]);
                }
                umma_commit(&acc_full[a]);
            }
        }
    } else {  // epilogue warps 2..9: TMEM lane quarter = warp % 4, column half = (warp - 2) / 4
        const int q = warp & 3, half = (warp - 2) >> 2;
        for (int j = 0; j < njobs; ++j) {
            const int a = j & 1;
            if (ok) ok = mbar_wait(&acc_full[a], (uint32_t)((j >> 1) & 1));
            ok = __all_sync(0xFFFFFFFFu, ok);  // tcgen05.ld is warp-collective
            if (!ok) break;
            tc_fence_after();
            const MlpJob jb = mlp_job(j, nb);
            const int gblk = (int)blockIdx.x + jb.blk * (int)gridDim.x;
            const int n0 = jb.h * TN;
            const bool l1 = jb.phase == 1;
            const float* sbias = l1 ? sb1 : sb2;
            // layer 1's rows of this warp: in scratch, or (training) in H1, where layer 2's rows go to H2 too
            const int grow0 = gblk * TM + q * 32;
            const int srow0 = train ? grow0 : scratch0 + (jb.blk & 1) * TM + q * 32;
            uint8_t* box = staging + (warp - 2) * MLP_STAGING;
            const uint32_t base = tmem + (uint32_t)(a * TN) + ((uint32_t)(q * 32) << 16);
            float z = 0.f;
            drain_accumulator<TN / 64>(base, half * (TN / 64), sbias + n0, [&](int c, const __nv_bfloat162* v) {
                if (l1) {
                    stage_chunk<2>(c, v, box, lane, &tmHst, n0, srow0);  // layer 1: rows to scratch / H1
                    if (h1bits) h1bits[ludax::h1bits_index(grow0 + lane, n0 + c * 32, MLP_N)] = nonzero_bits(v);
                } else {
                    z += dot_chunk(v, sw3 + n0 + c * 32);  // layer 2: the head's dot product
                    if (train) stage_chunk<2>(c, v, box, lane, &tmH2, n0, grow0);
                }
            });
            if (!l1) zpart[((size_t)gblk * TM + q * 32 + lane) * 4 + jb.h * 2 + half] = z;
            tc_fence_before();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(saddr(&acc_empty[a])) : "memory");
            if (l1 && jb.h == 1 && lane == 0) {  // both halves of this warp's rows are in global memory
                tma_store_wait_all();
                fence_proxy_async_global();
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(saddr(&h1_ready[jb.blk & 1]))
                             : "memory");
            }
        }
    }
    if (!ok) atomicOr(&g_umma_error, 1);
    if (warp >= 2 && lane == 0) tma_store_wait_all();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS));
}

// ------------------------------------------------------ backward GEMMs --
// The value net's backward contractions on the same pipeline (one TMA
// producer warp, one MMA warp, four epilogue warps, two TMEM accumulators),
// with operands that are K-major as above or MN-major: stored as K rows of M
// (or N) contiguous elements, which is how activations and gradients
// [batch][unit] look when the contraction runs over the batch.
//   GRAD_MASK    : out = bf16(mask > 0 ? A . B : 0) -- dZ1 = (dZ2 . W2) *
//                  [H1 > 0] with A = dZ2 K-major and B = W2 MN-major; with
//                  colpart given, also the column sums of the stored values
//                  (db1 = sum_b dZ1): each epilogue warp reads every staging
//                  box it fills back column-wise (lane l: columns 2l, 2l+1),
//                  keeps those running sums over all its tiles (the grid is a
//                  multiple of N / 256, so a CTA's tiles share their
//                  columns) and writes them once, as row (CTA / (N / 256)) *
//                  4 + warp of colpart [rows][N];
//   GRAD_MASKBITS: the same with the mask given as bits (h1bits_index
//                  layout): each epilogue lane loads its row's words of the
//                  tile before waiting for the accumulator, no mask tile is
//                  staged, and the ring has four stages;
//   GRAD_PARTIAL : part[split][m][n] = FP32 sum over the split's share of K
//                  of A[k][m] B[k][n] -- dW2 = dZ2^T . H1 and dW1 = dZ1^T . X,
//                  both operands MN-major; the batch is split so that
//                  (tiles x splits) work units fill the SMs, and the host sums
//                  the partials in a fixed order.
// An MN-major operand tile arrives as 64 x 64 boxes (64 K rows of 128
// bytes, 128-byte swizzle), box h holding elements 64 h .. 64 h + 63 along M
// (or N): in its shared-memory descriptor the leading byte offset is the
// 8 KB step between those 64-element blocks and the stride byte offset the
// 1 KB step between 8-row groups along K; each K = 16 MMA step moves the
// start by two groups.  GRAD_MASK stages the mask tile of each epilogue warp
// (its 32 rows x 256 columns) in shared memory with cp.async while the
// tile's MMAs run, rows XOR-swizzled by 16-byte chunk so the per-row reads
// are conflict-free; with that buffer the ring has three stages.
enum { GRAD_MASK = 0, GRAD_PARTIAL = 1, GRAD_MASKBITS = 2 };
constexpr int MN_BOX = 64 * TK * 2;  // one 64 (M or N) x 64 (K) BF16 box
constexpr int MASK_WARP_BYTES = 32 * TN * 2;
template <int EPI>
struct GradCfg {
    static constexpr int stages = EPI == GRAD_MASK ? 3 : DENSE_STAGES;
    static constexpr size_t smem = 1024 + (size_t)stages * STAGE + 4 * BOX_BYTES + 256 +
                                   (EPI == GRAD_MASK ? 4 * (size_t)MASK_WARP_BYTES : 0);
};

__device__ __forceinline__ uint64_t sw128_mn_desc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)(MN_BOX >> 4) << 16;                // leading byte offset: next 64-element block along M / N
    d |= (uint64_t)(1024 >> 4) << 32;                  // stride byte offset: next 8-row group along K
    d |= (uint64_t)1 << 46;                            // descriptor version
    d |= (uint64_t)2 << 61;                            // 128-byte swizzle
    return d;
}

template <bool A_MN, bool B_MN>
__device__ __forceinline__ void umma_bf16_major(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    // bits 15 / 16 of the instruction descriptor: A / B MN-major
    constexpr uint32_t idesc = kIdesc | (A_MN ? (1u << 15) : 0u) | (B_MN ? (1u << 16) : 0u);
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Column sums of a completed 32-row x 64-column BF16 staging box (the
// 128-byte-swizzle layout stage_chunk writes): lane l adds columns 2l and
// 2l + 1 down the 32 rows into a0, a1, in row order.  Each row is one
// 4-byte shared load per lane; a row's 16-byte chunks sit at chunk ^ (row
// % 8), so the 32 lanes of a row read 32 distinct banks.
__device__ __forceinline__ void box_colsum(const uint8_t* box, int lane, float& a0, float& a1) {
#pragma unroll 8
    for (int r = 0; r < 32; ++r) {
        const uint32_t u =
            *reinterpret_cast<const uint32_t*>(box + r * (OUT_BOX * 2) + (((lane >> 2) ^ (r & 7)) * 16) + (lane & 3) * 4);
        a0 += __uint_as_float(u << 16);
        a1 += __uint_as_float(u & 0xFFFF0000u);
    }
}

// 32-column chunks c0 .. c0 + NCH - 1 of one accumulator as raw FP32 bits:
// fn(c, x) with this lane's 32 values; the next chunk's load is in flight
// while fn runs.
template <int NCH, class F>
__device__ __forceinline__ void drain_raw(uint32_t base, F&& fn) {
    uint32_t r[2][32];
    tmem_ld32_async(base, r[0]);
    tmem_wait_ld(r[0]);
#pragma unroll
    for (int i = 0; i < NCH; ++i) {
        if (i + 1 < NCH) tmem_ld32_async(base + (uint32_t)((i + 1) * 32), r[(i + 1) & 1]);
        fn(i, r[i & 1]);
        if (i + 1 < NCH) tmem_wait_ld(r[(i + 1) & 1]);
    }
}

__device__ __forceinline__ void cp_async16_shared(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}

template <bool A_MN, bool B_MN, int EPI>
__global__ void __launch_bounds__(UMMA_THREADS, 1)
    umma_grad_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                     const __grid_constant__ CUtensorMap tmOut, int M, int N, int kblocks, int splits,
                     const __nv_bfloat16* __restrict__ mask, int ldm, float* __restrict__ part,
                     float* __restrict__ colpart, int last_use) {
    ludax::pdl_wait();
    constexpr int NS = GradCfg<EPI>::stages;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t* staging = smem + NS * STAGE;
    uint8_t* smask = staging + 4 * BOX_BYTES;  // GRAD_MASK: four warps' mask tiles (GRAD_MASKBITS: read from global)
    uint64_t* full = reinterpret_cast<uint64_t*>(smask + (EPI == GRAD_MASK ? 4 * MASK_WARP_BYTES : 0));
    uint64_t* empty = full + NS;
    uint64_t* acc_full = empty + NS;    // [2] MMA -> epilogue
    uint64_t* acc_empty = acc_full + 2;  // [2] epilogue -> MMA
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntn = N / TN, tiles = (M / TM) * ntn, units = tiles * splits;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&acc_full[a], 1);
            mbar_init(&acc_empty[a], 128);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(saddr(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;
    // work unit u: tile u % tiles over K blocks [kb0, kb1) of split u / tiles
    auto unit = [&](int u, int& m0, int& n0, int& sp, int& kb0, int& kb1) {
        const int tile = u % tiles;
        sp = u / tiles;
        m0 = (tile / ntn) * TM;
        n0 = (tile % ntn) * TN;
        kb0 = (int)((long long)sp * kblocks / splits);
        kb1 = (int)((long long)(sp + 1) * kblocks / splits);
    };

    if (warp == 0) {
        if (lane == 0) {  // TMA producer
            // operands read for the last time in the step (last_use bit 0: A, bit 1: B) leave L2 first
            const uint64_t pa = (last_use & 1) ? l2_last_use_policy() : 0ull;
            const uint64_t pb = (last_use & 2) ? l2_last_use_policy() : 0ull;
            int it = 0;
            for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
                int m0, n0, sp, kb0, kb1;
                unit(u, m0, n0, sp, kb0, kb1);
                for (int kt = kb0; kt < kb1 && ok; ++kt, ++it) {
                    const int s = it % NS;
                    if (it >= NS) ok = mbar_wait(&empty[s], (uint32_t)(((it / NS) & 1) ^ 1));
                    if (!ok) break;
                    uint8_t* st = smem + s * STAGE;
                    mbar_expect_tx(&full[s], STAGE);
                    if (A_MN) {
#pragma unroll
                        for (int h = 0; h < TM / 64; ++h)
                            tma_load_2d_pol(st + h * MN_BOX, &tmA, &full[s], m0 + 64 * h, kt * TK, pa);
                    } else {
                        tma_load_2d_pol(st, &tmA, &full[s], kt * TK, m0, pa);
                    }
                    if (B_MN) {
#pragma unroll
                        for (int h = 0; h < TN / 64; ++h)
                            tma_load_2d_pol(st + A_TILE + h * MN_BOX, &tmB, &full[s], n0 + 64 * h, kt * TK, pb);
                    } else {
                        tma_load_2d_pol(st + A_TILE, &tmB, &full[s], kt * TK, n0, pb);
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            int it = 0, local = 0;
            for (int u = blockIdx.x; u < units && ok; u += gridDim.x, ++local) {
                int m0, n0, sp, kb0, kb1;
                unit(u, m0, n0, sp, kb0, kb1);
                const int a = local & 1;
                if (local >= 2) ok = mbar_wait(&acc_empty[a], (uint32_t)(((local >> 1) & 1) ^ 1));
                if (!ok) break;
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(a * TN);
                for (int kt = kb0; kt < kb1 && ok; ++kt, ++it) {
                    const int s = it % NS;
                    ok = mbar_wait(&full[s], (uint32_t)((it / NS) & 1));
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t sa = saddr(smem + s * STAGE);
                    const uint64_t ad = A_MN ? sw128_mn_desc(sa) : sw128_desc(sa);
                    const uint64_t bd = B_MN ? sw128_mn_desc(sa + A_TILE) : sw128_desc(sa + A_TILE);
                    constexpr uint64_t astep = A_MN ? (2048 >> 4) : 2, bstep = B_MN ? (2048 >> 4) : 2;
#pragma unroll
                    for (int kk = 0; kk < TK / 16; ++kk)
                        umma_bf16_major<A_MN, B_MN>(d, ad + astep * kk, bd + bstep * kk, (kt != kb0 || kk) ? 1u : 0u);
                    umma_commit(&empty[s]);
                }
                umma_commit(&acc_full[a]);
            }
        }
    } else {  // epilogue warps 2..5: TMEM lane quarter = warp % 4
        const int q = warp & 3;
        uint8_t* wmask = smask + q * MASK_WARP_BYTES;
        float csum[TN / 32];  // GRAD_MASK with colpart: columns 64 b + 2 lane, + 1 of box b, summed over the tiles
#pragma unroll
        for (int c = 0; c < TN / 32; ++c) csum[c] = 0.f;
        int local = 0;
        for (int u = blockIdx.x; u < units; u += gridDim.x, ++local) {
            int m0, n0, sp, kb0, kb1;
            unit(u, m0, n0, sp, kb0, kb1);
            const int row0 = m0 + q * 32;
            if (EPI == GRAD_MASK) {  // this warp's 32 mask rows, 16 bytes per lane per row, while the MMAs run
                __syncwarp();        // every lane is done reading the previous tile's rows
                const uint32_t wm = saddr(wmask);
                for (int r = 0; r < 32; ++r)
                    cp_async16_shared(wm + (uint32_t)(r * (TN * 2) + ((lane ^ (r & 7)) * 16)),
                                      mask + (size_t)(row0 + r) * ldm + n0 + lane * 8);
                asm volatile("cp.async.commit_group;\n" ::: "memory");
            }
            uint32_t mw[TN / 32];  // GRAD_MASKBITS: this lane's mask word of each 32-column chunk, fetched before the wait
            if (EPI == GRAD_MASKBITS) {
                const uint32_t* bits = reinterpret_cast<const uint32_t*>(mask);
#pragma unroll
                for (int c = 0; c < TN / 32; ++c) mw[c] = bits[ludax::h1bits_index(row0 + lane, n0 + c * 32, N)];
            }
            const int a = local & 1;
            if (ok) ok = mbar_wait(&acc_full[a], (uint32_t)((local >> 1) & 1));
            ok = __all_sync(0xFFFFFFFFu, ok);  // tcgen05.ld is warp-collective
            if (!ok) break;
            tc_fence_after();
            if (EPI == GRAD_MASK) {
                asm volatile("cp.async.wait_group 0;\n" ::: "memory");
                __syncwarp();
            }
            const uint32_t base = tmem + (uint32_t)(a * TN) + ((uint32_t)(q * 32) << 16);
            drain_raw<TN / 32>(base, [&](int c, const uint32_t* x) {
                if (EPI == GRAD_PARTIAL) {
                    float4* dst = reinterpret_cast<float4*>(part + ((size_t)sp * M + row0 + lane) * N + n0 + c * 32);
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        dst[j] = make_float4(__uint_as_float(x[4 * j]), __uint_as_float(x[4 * j + 1]),
                                             __uint_as_float(x[4 * j + 2]), __uint_as_float(x[4 * j + 3]));
                } else {
                    __align__(16) __nv_bfloat162 v[16];
                    if (EPI == GRAD_MASKBITS) {
                        const uint32_t m = mw[c];
#pragma unroll
                        for (int k = 0; k < 16; ++k)
                            v[k] = __floats2bfloat162_rn((m >> (2 * k)) & 1u ? __uint_as_float(x[2 * k]) : 0.f,
                                                         (m >> (2 * k + 1)) & 1u ? __uint_as_float(x[2 * k + 1]) : 0.f);
                    } else {
                        const uint8_t* myrow = wmask + lane * (TN * 2);
#pragma unroll
                        for (int j = 0; j < 4; ++j) {  // 16-byte chunk 4 c + j of this lane's mask row
                            const uint4 m4 = *reinterpret_cast<const uint4*>(myrow + (((4 * c + j) ^ (lane & 7)) * 16));
                            const __nv_bfloat162* mk = reinterpret_cast<const __nv_bfloat162*>(&m4);
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const float2 mf = __bfloat1622float2(mk[e]);
                                const int i = 8 * j + 2 * e;
                                v[4 * j + e] = __floats2bfloat162_rn(mf.x > 0.f ? __uint_as_float(x[i]) : 0.f,
                                                                     mf.y > 0.f ? __uint_as_float(x[i + 1]) : 0.f);
                            }
                        }
                    }
                    stage_chunk<1>(c, v, staging + q * BOX_BYTES, lane, &tmOut, n0, row0);
                    // a full box (its store just issued reads it too; the box is
                    // refilled only after the store has read it and this warp moved on)
                    if (colpart && (c & 1)) box_colsum(staging + q * BOX_BYTES, lane, csum[c - 1], csum[c]);
                }
            });
            tc_fence_before();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(saddr(&acc_empty[a])) : "memory");
        }
        if (EPI == GRAD_MASK) asm volatile("cp.async.wait_group 0;\n" ::: "memory");  // nothing in flight at exit
        if (EPI != GRAD_PARTIAL) {
            if (colpart) {
                float* dst = colpart + (size_t)((blockIdx.x / ntn) * 4 + q) * N + (blockIdx.x % ntn) * TN + 2 * lane;
#pragma unroll
                for (int b = 0; b < TN / 64; ++b) *reinterpret_cast<float2*>(dst + b * 64) = make_float2(csum[2 * b], csum[2 * b + 1]);
            }
        }
    }
    if (!ok) atomicOr(&g_umma_error, 1);
    if (warp >= 2 && lane == 0) tma_store_wait_all();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS));
}

// ------------------------------------------------------ wait self-test --
// The failure path of the bounded waits, exercised without a fault: one
// thread waits on an mbarrier that nothing will ever arrive at, gives up
// after `limit` clock cycles and records the expiry in the device error word
// (bit 2), exactly as the GEMM kernels do when a pipeline stage never lands.
__global__ void wait_selftest_kernel(long long limit) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const long long t0 = clock64();
    bool done = false;
    while (!(done = mbar_try_wait(&bar, 0u)))
        if (clock64() - t0 > limit) break;
    if (!done) atomicOr(&g_umma_error, 2);
}

// ------------------------------------------------------------ host side --
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
    static EncodeTiled fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    });
    return fn;
}

// 2-D BF16 tensor map over a row-major [rows][cols] matrix (row pitch ld
// elements) with a box of box_rows x 64 columns and 128-byte swizzle.
bool make_map(CUtensorMap* m, const void* base, int rows, int cols, int box_rows, int ld) {
    EncodeTiled fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};  // 64 BF16 = the 128-byte swizzle span
    cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

namespace ludax {

// A kernel's dynamic shared-memory limit is an attribute of the function on
// the current device: set once per (kernel, device), under a lock.
int ensure_smem_limit(const void* kernel, size_t bytes) {
    static std::mutex mu;
    static std::set<std::pair<const void*, int>> done;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LUDAX_ERR_CUDA;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({kernel, dev})) return LUDAX_OK;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
        return LUDAX_ERR_CUDA;
    done.insert({kernel, dev});
    return LUDAX_OK;
}

// SMs of the current device (0 on error)
int device_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return sms;
}

bool umma_dense_supported(int M, int N, int K) {
    return M > 0 && N > 0 && K > 0 && M % TM == 0 && N % TN == 0 && K % TK == 0 && N <= MAX_N;
}

int umma_dense_relu(const void* A, const void* B, const float* bias, void* out, int M, int N, int K, int ldo,
                    cudaStream_t s) {
    return umma_dense_relu_ex(A, K, B, K, bias, out, ldo, nullptr, nullptr, M, N, K, s);
}

int umma_dense_relu_ex(const void* A, int lda, const void* B, int ldb, const float* bias, void* out, int ldo,
                       const void* w3, float* zpart, int M, int N, int K, cudaStream_t s) {
    const bool head = w3 != nullptr, store = out != nullptr;
    if (!umma_dense_supported(M, N, K) || lda < K || ldb < K || lda % 8 || ldb % 8 || ((uintptr_t)A % 16) ||
        ((uintptr_t)B % 16))
        return LUDAX_ERR_SIZE;
    if ((!head && !store) || (head && !zpart) || (store && (ldo % 8 || ((uintptr_t)out % 16)))) return LUDAX_ERR_SIZE;
    CUtensorMap ma, mb, mo;
    // with nothing stored the output map is a valid placeholder over A
    if (!make_map(&ma, A, M, K, TM, lda) || !make_map(&mb, B, N, K, TN, ldb) ||
        !(store ? make_map(&mo, out, M, N, 32, ldo) : make_map(&mo, A, M, K, 32, lda)))
        return LUDAX_ERR_CUDA;
    const int sms = device_sms();
    if (!sms || ensure_smem_limit((const void*)umma_dense_relu_kernel, UMMA_SMEM)) return LUDAX_ERR_CUDA;
    const int ntiles = (M / TM) * (N / TN);
    const int grid = ntiles < sms ? ntiles : sms;
    return launch_dependent(umma_dense_relu_kernel, (unsigned)grid, UMMA_THREADS, UMMA_SMEM, s, ma, mb, mo, M, N, K,
                            bias, static_cast<const __nv_bfloat16*>(w3), zpart, store ? 1 : 0) == cudaSuccess
               ? LUDAX_OK
               : LUDAX_ERR_CUDA;
}

// grid of a backward launch: one CTA per SM at most, a multiple of the
// column tiles N / 256 (so a persistent CTA's tiles all cover the same
// columns; there are always at least that many units)
static int grad_grid(int units, int ntn, int sms) {
    int g = units < sms ? units : sms;
    g -= g % ntn;
    return g < ntn ? ntn : g;
}

template <bool A_MN, bool B_MN, int EPI>
static int launch_grad(const CUtensorMap& ma, const CUtensorMap& mb, const CUtensorMap& mo, int M, int N, int kblocks,
                       int splits, const void* mask, int ldm, float* part, float* colpart, int sms, cudaStream_t s,
                       int last_use) {
    auto k = umma_grad_kernel<A_MN, B_MN, EPI>;
    if (ensure_smem_limit((const void*)k, GradCfg<EPI>::smem)) return LUDAX_ERR_CUDA;
    const int units = (M / TM) * (N / TN) * splits;
    return launch_dependent(k, (unsigned)grad_grid(units, N / TN, sms), UMMA_THREADS, GradCfg<EPI>::smem, s, ma, mb,
                            mo, M, N, kblocks, splits, static_cast<const __nv_bfloat16*>(mask), ldm, part,
                            colpart, last_use) == cudaSuccess
               ? LUDAX_OK
               : LUDAX_ERR_CUDA;
}

int umma_grad_colrows(int M, int N) {
    const int sms = device_sms();
    if (!sms || !umma_dense_supported(M, N, TK)) return 0;
    return grad_grid((M / TM) * (N / TN), N / TN, sms) / (N / TN) * 4;
}

int umma_grad_mask(const void* A, const void* B, const void* mask, void* out, int M, int N, int K, float* colpart,
                   cudaStream_t s) {
    if (!umma_dense_supported(M, N, K) || !A || !B || !mask || !out || N % 8 || K % 8 || ((uintptr_t)A % 16) ||
        ((uintptr_t)B % 16) || ((uintptr_t)mask % 16) || ((uintptr_t)out % 16))
        return LUDAX_ERR_SIZE;
    const int sms = device_sms();
    if (!sms) return LUDAX_ERR_CUDA;
    CUtensorMap ma, mb, mo;
    // A [M][K] K-major; B [K][N] MN-major (64 x 64 boxes); out [M][N] in 32-row boxes
    if (!make_map(&ma, A, M, K, TM, K) || !make_map(&mb, B, K, N, 64, N) || !make_map(&mo, out, M, N, 32, N))
        return LUDAX_ERR_CUDA;
    if (colpart && ((uintptr_t)colpart % 8)) return LUDAX_ERR_SIZE;
    return launch_grad<false, true, GRAD_MASK>(ma, mb, mo, M, N, K / TK, 1, mask, N, nullptr, colpart, sms, s, 1);
}

int umma_grad_maskbits(const void* A, const void* B, const uint32_t* maskbits, void* out, int M, int N, int K,
                       float* colpart, cudaStream_t s) {
    if (!umma_dense_supported(M, N, K) || !A || !B || !maskbits || !out || N % 8 || K % 8 || ((uintptr_t)A % 16) ||
        ((uintptr_t)B % 16) || ((uintptr_t)maskbits % 4) || ((uintptr_t)out % 16))
        return LUDAX_ERR_SIZE;
    const int sms = device_sms();
    if (!sms) return LUDAX_ERR_CUDA;
    CUtensorMap ma, mb, mo;
    if (!make_map(&ma, A, M, K, TM, K) || !make_map(&mb, B, K, N, 64, N) || !make_map(&mo, out, M, N, 32, N))
        return LUDAX_ERR_CUDA;
    if (colpart && ((uintptr_t)colpart % 8)) return LUDAX_ERR_SIZE;
    return launch_grad<false, true, GRAD_MASKBITS>(ma, mb, mo, M, N, K / TK, 1, maskbits, N, nullptr, colpart, sms,
                                                   s, 1);
}

int umma_grad_weights(const void* A, int lda, const void* B, int ldb, int M, int N, int K, float* part,
                      long long part_floats, int* splits_out, cudaStream_t s, int last_use) {
    if (!umma_dense_supported(M, N, K) || !A || !B || !part || !splits_out || lda < M || ldb < N || lda % 8 ||
        ldb % 8 || ((uintptr_t)A % 16) || ((uintptr_t)B % 16) || ((uintptr_t)part % 16))
        return LUDAX_ERR_SIZE;
    const int sms = device_sms();
    if (!sms) return LUDAX_ERR_CUDA;
    const int tiles = (M / TM) * (N / TN), kblocks = K / TK;
    long long splits = sms / tiles;          // enough work units to fill the SMs (one when the tiles already do)
    if (splits > kblocks) splits = kblocks;  // every split gets at least one K block
    if (splits > part_floats / ((long long)M * N)) splits = part_floats / ((long long)M * N);
    if (splits < 1) splits = 1;
    if ((long long)M * N > part_floats) return LUDAX_ERR_SIZE;  // not even one partial fits
    CUtensorMap ma, mb;
    // A [K][M] and B [K][N], both MN-major (64 x 64 boxes); nothing is stored through a tensor map
    if (!make_map(&ma, A, K, M, 64, lda) || !make_map(&mb, B, K, N, 64, ldb)) return LUDAX_ERR_CUDA;
    *splits_out = (int)splits;
    return launch_grad<true, true, GRAD_PARTIAL>(ma, mb, ma, M, N, kblocks, (int)splits, nullptr, 0, part, nullptr,
                                                 sms, s, last_use);
}

int umma_mlp_scratch_rows() { return device_sms() * 2 * TM; }

int umma_mlp_head(const void* X, int ldx, int K1, const void* W1, int ldw1, const float* b1, const void* W2,
                  const float* b2, const void* w3, float* zpart, void* scratch, int scratch_rows, int M,
                  cudaStream_t s) {
    if (M <= 0 || M % TM || K1 <= 0 || K1 % TK || K1 > ldx || K1 > ldw1 || ldx % 8 || ldw1 % 8 || !zpart ||
        !scratch || ((uintptr_t)X % 16) || ((uintptr_t)W1 % 16) || ((uintptr_t)W2 % 16) || ((uintptr_t)scratch % 16))
        return LUDAX_ERR_SIZE;
    const int sms = device_sms();
    if (!sms) return LUDAX_ERR_CUDA;
    const int nblk = M / TM, grid = nblk < sms ? nblk : sms;
    if (scratch_rows < grid * 2 * TM) return LUDAX_ERR_SIZE;
    CUtensorMap mx, mw1, mhs, mhl, mw2;
    if (!make_map(&mx, X, M, K1, TM, ldx) || !make_map(&mw1, W1, MLP_N, K1, TN, ldw1) ||
        !make_map(&mhs, scratch, scratch_rows, MLP_N, 32, MLP_N) || !make_map(&mhl, scratch, scratch_rows, MLP_N, TM, MLP_N) ||
        !make_map(&mw2, W2, MLP_N, MLP_N, TN, MLP_N))
        return LUDAX_ERR_CUDA;
    if (ensure_smem_limit((const void*)umma_mlp_head_kernel, MLP_SMEM)) return LUDAX_ERR_CUDA;
    // no H2 is stored: its map is a valid placeholder over the scratch
    return launch_dependent(umma_mlp_head_kernel, (unsigned)grid, MLP_THREADS, MLP_SMEM, s, mx, mw1, mhs, mhl, mw2, mhs,
                            M, K1, b1, b2, static_cast<const __nv_bfloat16*>(w3), zpart, 0,
                            static_cast<uint32_t*>(nullptr)) == cudaSuccess
               ? LUDAX_OK
               : LUDAX_ERR_CUDA;
}

int umma_mlp_train(const void* X, int ldx, int K1, const void* W1, int ldw1, const float* b1, const void* W2,
                   const float* b2, const void* w3, float* zpart, void* H1, void* H2, uint32_t* h1bits, int M,
                   cudaStream_t s) {
    if (M <= 0 || M % TM || K1 <= 0 || K1 % TK || K1 > ldx || K1 > ldw1 || ldx % 8 || ldw1 % 8 || !zpart || !H1 ||
        !H2 || ((uintptr_t)X % 16) || ((uintptr_t)W1 % 16) || ((uintptr_t)W2 % 16) || ((uintptr_t)H1 % 16) ||
        ((uintptr_t)H2 % 16))
        return LUDAX_ERR_SIZE;
    const int sms = device_sms();
    if (!sms) return LUDAX_ERR_CUDA;
    const int nblk = M / TM, grid = nblk < sms ? nblk : sms;
    CUtensorMap mx, mw1, mhs, mhl, mw2, mh2;
    if (!make_map(&mx, X, M, K1, TM, ldx) || !make_map(&mw1, W1, MLP_N, K1, TN, ldw1) ||
        !make_map(&mhs, H1, M, MLP_N, 32, MLP_N) || !make_map(&mhl, H1, M, MLP_N, TM, MLP_N) ||
        !make_map(&mw2, W2, MLP_N, MLP_N, TN, MLP_N) || !make_map(&mh2, H2, M, MLP_N, 32, MLP_N))
        return LUDAX_ERR_CUDA;
    if (ensure_smem_limit((const void*)umma_mlp_head_kernel, MLP_SMEM)) return LUDAX_ERR_CUDA;
    return launch_dependent(umma_mlp_head_kernel, (unsigned)grid, MLP_THREADS, MLP_SMEM, s, mx, mw1, mhs, mhl, mw2, mh2,
                            M, K1, b1, b2, static_cast<const __nv_bfloat16*>(w3), zpart, 1, h1bits) == cudaSuccess
               ? LUDAX_OK
               : LUDAX_ERR_CUDA;
}

}  // namespace ludax

extern "C" {

int ludax_dense_bf16_relu(const uint16_t* a_dev, const uint16_t* b_dev, const float* bias_dev, uint16_t* out_dev,
                          int32_t M, int32_t N, int32_t K, int32_t ld_out, void* stream) {
    ludax::ApiRange api_range("ludax_dense_bf16_relu");
    if (!a_dev || !b_dev || !bias_dev || !out_dev) return LUDAX_ERR_ARG;
    return ludax::umma_dense_relu(a_dev, b_dev, bias_dev, out_dev, M, N, K, ld_out, (cudaStream_t)stream);
}

int ludax_selftest_wait(int64_t limit_cycles, void* stream) {
    if (limit_cycles < 1 || limit_cycles > kWaitLimit) return LUDAX_ERR_ARG;
    wait_selftest_kernel<<<1, 32, 0, (cudaStream_t)stream>>>((long long)limit_cycles);
    return cudaGetLastError() == cudaSuccess ? LUDAX_OK : LUDAX_ERR_CUDA;
}

int ludax_device_error(int32_t* error_out) {
    int h = 0, z = 0;
    if (cudaMemcpyFromSymbol(&h, g_umma_error, sizeof(int)) != cudaSuccess ||
        cudaMemcpyToSymbol(g_umma_error, &z, sizeof(int)) != cudaSuccess)
        return LUDAX_ERR_CUDA;
    if (error_out) *error_out = h;
    return h ? LUDAX_ERR_TIMEOUT : LUDAX_OK;
}

}  // extern "C"
