// ludax_net.cu -- the value network that truncates playouts: BF16 MLP
// (inputs [P1 plane, P2 plane, side to move] -> 512 ReLU -> 512 ReLU -> tanh),
// FP32 accumulation, hand-written forward, backward and Adam kernels, input
// packing from env state, and the truncated value estimator (a few random
// plies, then the net).
//
// Precision: weights live as FP32 masters with BF16 copies used by every
// GEMM; activations H1, H2 and the hidden-layer gradients dZ2, dZ1 are stored
// in BF16; every product accumulates in FP32; the output layer, loss,
// gradient reductions and Adam run in FP32.
//
// GEMMs run on the tensor cores: one templated kernel computes
// C[m][n] = sum_k A(m,k) B(n,k) over 128x128 tiles with BK = 32, three
// cp.async stages, ldmatrix (transposing where an operand is stored
// M- or N-major) and mma.m16n8k16 BF16 -> FP32, with a fused epilogue.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "ludax_internal.cuh"

using namespace ludax;

namespace {

constexpr int kH = 512;  // hidden width
constexpr int BM = 128, BN = 128, BKT = 32, STAGES = 3, GEMM_THREADS = 256;
constexpr int KMAJ_LD = BKT + 8;   // smem row length of a K-major tile (halves)
constexpr int MMAJ_LD = BM + 8;    // smem row length of an M/N-major tile (halves)
constexpr int TILE_HALVES = (BM * KMAJ_LD > BKT * MMAJ_LD) ? BM * KMAJ_LD : BKT * MMAJ_LD;
constexpr size_t GEMM_SMEM = sizeof(__nv_bfloat16) * TILE_HALVES * 2 * STAGES;

enum { EPI_BIAS_RELU = 0, EPI_MASK = 1, EPI_PARTIAL = 2 };

struct GemmArgs {
    const __nv_bfloat16* A;
    const __nv_bfloat16* B;
    int M, N, K, lda, ldb, k_per_split;
    const float* bias;          // EPI_BIAS_RELU: [N]
    const __nv_bfloat16* mask;  // EPI_MASK: [M][ldo], multiply by (mask > 0)
    __nv_bfloat16* out;         // EPI_BIAS_RELU / EPI_MASK: [M][ldo]
    int ldo;
    float* partial;             // EPI_PARTIAL: [splits][M][N]
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldsm_x4(uint32_t* r, const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t* r, const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Copy one BK-deep stage of an operand tile into shared memory.
//   KMAJOR: global X[row][k] (row = m or n), tile sm[row][k] with row length KMAJ_LD
//   else  : global X[k][row],               tile sm[k][row] with row length MMAJ_LD
template <bool KMAJOR>
__device__ __forceinline__ void load_tile(__nv_bfloat16* sm, const __nv_bfloat16* g, int ld, int row0, int k0) {
    const int t = threadIdx.x;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        int c = t + i * GEMM_THREADS;  // 512 chunks of 8 halves
        if (KMAJOR) {
            int r = c >> 2, kc = (c & 3) * 8;
            cp_async16(sm + r * KMAJ_LD + kc, g + (size_t)(row0 + r) * ld + k0 + kc);
        } else {
            int r = c >> 4, mc = (c & 15) * 8;
            cp_async16(sm + r * MMAJ_LD + mc, g + (size_t)(k0 + r) * ld + row0 + mc);
        }
    }
}

template <bool AK, bool BK_, int EPI>
__global__ void __launch_bounds__(GEMM_THREADS) gemm_bf16_kernel(GemmArgs g) {
    extern __shared__ __align__(16) __nv_bfloat16 gsm[];
    __nv_bfloat16* sA = gsm;
    __nv_bfloat16* sB = gsm + TILE_HALVES * STAGES;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kbeg = blockIdx.z * g.k_per_split;
    const int ktiles = g.k_per_split / BKT;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = warp >> 2, wn = warp & 3;  // 2 x 4 warps, warp tile 64 x 32

    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

    auto issue = [&](int kt) {
        int s = kt % STAGES;
        load_tile<AK>(sA + s * TILE_HALVES, g.A, g.lda, m0, kbeg + kt * BKT);
        load_tile<BK_>(sB + s * TILE_HALVES, g.B, g.ldb, n0, kbeg + kt * BKT);
    };
#pragma unroll
    for (int s = 0; s < STAGES - 1; ++s) {
        if (s < ktiles) issue(s);
        cp_async_commit();
    }
    for (int kt = 0; kt < ktiles; ++kt) {
        cp_async_wait<STAGES - 2>();
        __syncthreads();
        if (kt + STAGES - 1 < ktiles) issue(kt + STAGES - 1);
        cp_async_commit();
        const __nv_bfloat16* a = sA + (kt % STAGES) * TILE_HALVES;
        const __nv_bfloat16* b = sB + (kt % STAGES) * TILE_HALVES;
#pragma unroll
        for (int kk = 0; kk < BKT; kk += 16) {
            uint32_t af[4][4], bfr[4][2];
#pragma unroll
            for (int mi = 0; mi < 4; ++mi) {
                int mr = wm * 64 + mi * 16;
                if (AK) {
                    ldsm_x4(af[mi], a + (mr + (lane & 15)) * KMAJ_LD + kk + (lane >> 4) * 8);
                } else {
                    ldsm_x4_t(af[mi], a + (kk + (lane & 7) + (lane >> 4) * 8) * MMAJ_LD + mr + ((lane >> 3) & 1) * 8);
                }
            }
#pragma unroll
            for (int nj = 0; nj < 2; ++nj) {
                int nr = wn * 32 + nj * 16;
                uint32_t r[4];
                if (BK_) {
                    ldsm_x4(r, b + (nr + (lane & 7) + (lane >> 4) * 8) * KMAJ_LD + kk + ((lane >> 3) & 1) * 8);
                } else {
                    ldsm_x4_t(r, b + (kk + (lane & 7) + ((lane >> 3) & 1) * 8) * MMAJ_LD + nr + (lane >> 4) * 8);
                }
                bfr[nj * 2][0] = r[0];
                bfr[nj * 2][1] = r[1];
                bfr[nj * 2 + 1][0] = r[2];
                bfr[nj * 2 + 1][1] = r[3];
            }
#pragma unroll
            for (int mi = 0; mi < 4; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], af[mi], bfr[ni]);
        }
    }
    cp_async_wait<0>();

    const int gid = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                int row = m0 + wm * 64 + mi * 16 + gid + h * 8;
                int col = n0 + wn * 32 + ni * 8 + tig * 2;
                float v0 = acc[mi][ni][2 * h], v1 = acc[mi][ni][2 * h + 1];
                if (EPI == EPI_BIAS_RELU) {
                    v0 = fmaxf(v0 + g.bias[col], 0.f);
                    v1 = fmaxf(v1 + g.bias[col + 1], 0.f);
                    *reinterpret_cast<__nv_bfloat162*>(g.out + (size_t)row * g.ldo + col) = __floats2bfloat162_rn(v0, v1);
                } else if (EPI == EPI_MASK) {
                    __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162*>(g.mask + (size_t)row * g.ldo + col);
                    v0 = __bfloat162float(mk.x) > 0.f ? v0 : 0.f;
                    v1 = __bfloat162float(mk.y) > 0.f ? v1 : 0.f;
                    *reinterpret_cast<__nv_bfloat162*>(g.out + (size_t)row * g.ldo + col) = __floats2bfloat162_rn(v0, v1);
                } else {
                    float* p = g.partial + (size_t)blockIdx.z * g.M * g.N + (size_t)row * g.N + col;
                    *reinterpret_cast<float2*>(p) = make_float2(v0, v1);
                }
            }
}

template <bool AK, bool BK_, int EPI>
int launch_gemm(const GemmArgs& a, int splits, cudaStream_t s) {
    if (a.M % BM || a.N % BN || a.K % (BKT * splits) || a.lda % 8 || a.ldb % 8) return LUDAX_ERR_SIZE;
    auto k = gemm_bf16_kernel<AK, BK_, EPI>;
    if (ensure_smem_limit((const void*)k, GEMM_SMEM)) return LUDAX_ERR_CUDA;
    GemmArgs g = a;
    g.k_per_split = a.K / splits;
    dim3 grid(a.N / BN, a.M / BM, splits);
    k<<<grid, GEMM_THREADS, GEMM_SMEM, s>>>(g);
    return cudaGetLastError() == cudaSuccess ? LUDAX_OK : LUDAX_ERR_CUDA;
}

// ------------------------------------------------------------ head layer --
// One warp per row: z = H2[b] . w3 + b3, v = tanh(z), p = (v + 1) / 2.  With
// labels: g3[b] = dL/dz for L = mean (p - y)^2, and the row's squared error.
__global__ void head_forward_kernel(const __nv_bfloat16* H2, const __nv_bfloat16* w3, const float* b3, int B,
                                    float* p_out, const float* y, float* g3, float* sqerr) {
    int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (row >= B) return;
    const uint4* h = reinterpret_cast<const uint4*>(H2 + (size_t)row * kH);
    const uint4* w = reinterpret_cast<const uint4*>(w3);
    float z = 0.f;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        uint4 hv = h[lane + 32 * i], wv = w[lane + 32 * i];
        const __nv_bfloat162* hp = reinterpret_cast<const __nv_bfloat162*>(&hv);
        const __nv_bfloat162* wp = reinterpret_cast<const __nv_bfloat162*>(&wv);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float2 a = __bfloat1622float2(hp[j]), c = __bfloat1622float2(wp[j]);
            z = fmaf(a.x, c.x, z);
            z = fmaf(a.y, c.y, z);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xFFFFFFFFu, z, o);
    if (lane == 0) {
        z += b3[0];
        float v = tanhf(z);
        float p = 0.5f * (v + 1.f);
        if (p_out) p_out[row] = p;
        if (y) {
            float d = p - y[row];
            g3[row] = d * (1.f - v * v) / (float)B;  // 2 (p-y)/B * (1/2) (1 - v^2)
            sqerr[row] = d * d;
        }
    }
}

// Row-chunk kernels over [B][kH] BF16 matrices: a 256-thread block takes
// HB_ROWS rows; its thread t covers columns 8 (t % 64) .. 8 (t % 64) + 7 of
// rows r0 + t / 64, r0 + t / 64 + 4, ... (16-byte loads, four rows in
// flight), and the four row groups' sums are added in a fixed order.  112
// rows make a 65,536-row batch 586 chunks, one wave of four resident blocks
// on each of 148 SMs (128 rows left 512 blocks spread 3 or 4 per SM).
constexpr int HB_ROWS = 112, HB_GROUPS = 4;
constexpr int HB_COLS = 2 * kH + 2;  // head partials per chunk: db2 | dw3 | db3 | squared error

__device__ __forceinline__ void load8(const __nv_bfloat16* p, float* f) {
    const uint4 v = *reinterpret_cast<const uint4*>(p);
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float2 x = __bfloat1622float2(h[e]);
        f[2 * e] = x.x;
        f[2 * e + 1] = x.y;
    }
}

// dZ2[b][j] = g3[b] w3[j] [H2[b][j] > 0] (stored bf16), plus the chunk's
// partials in row blockIdx.x of part[chunks][HB_COLS]: db2 = sum_b dZ2
// (unrounded), dw3 = sum_b g3 H2, db3 = sum_b g3 and the summed squared
// error -- b2, w3, b3 in the order the gradient vector stores them.
// With zpart given (the training forward's fused head: zparts partial dot
// products per row) the row's g3 and squared error are formed here from z, y and b3,
// as head_finish_kernel does; otherwise they are read from g3 / sqerr.
constexpr int ZPARTS = 4;  // head partials per row of the one-launch training forward (umma_mlp_train)
__device__ __forceinline__ void head_row(const float* zpart, int parts, const float* y, const float* b3, int B,
                                         int r, float& g, float& se) {
    float z = 0.f;
    for (int i = 0; i < parts; ++i) z += zpart[(size_t)r * parts + i];
    const float v = tanhf(z + b3[0]), p = 0.5f * (v + 1.f), d = p - y[r];
    g = d * (1.f - v * v) / (float)B;  // 2 (p-y)/B * (1/2) (1 - v^2)
    se = d * d;
}
// A 16-byte global load whose line L2 may give up first: for data read for
// the last time (H2 in the head's backward), so that the rows written next
// (dZ2, read by the next two launches) keep their place.
__device__ __forceinline__ uint4 ld_last_use(const void* a) {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
    uint4 v;
    asm volatile("ld.global.L2::cache_hint.v4.b32 {%0, %1, %2, %3}, [%4], %5;\n"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(a), "l"(pol)
                 : "memory");
    return v;
}
__global__ void __launch_bounds__(256) head_backward_kernel(const __nv_bfloat16* H2, const __nv_bfloat16* w3,
                                                            const float* g3, const float* sqerr, const float* zpart,
                                                            int zparts, const float* y, const float* b3, int B,
                                                            __nv_bfloat16* dZ2, float* part) {
    pdl_wait();
    __shared__ float sh[HB_GROUPS - 1][HB_COLS];
    __shared__ float sg[HB_ROWS], ss[HB_ROWS];  // the chunk's rows: g3 and squared error
    const int grp = threadIdx.x >> 6, j0 = (threadIdx.x & 63) * 8;
    const bool first = (threadIdx.x & 63) == 0;
    float w[8], ab[8], aw[8], ag = 0.f, al = 0.f;
    load8(w3 + j0, w);
#pragma unroll
    for (int e = 0; e < 8; ++e) ab[e] = aw[e] = 0.f;
    const int r0 = blockIdx.x * HB_ROWS, r1 = min(r0 + HB_ROWS, B);
    // the thread's first HB_PRE rows of H2 are fetched first, so that their
    // loads overlap the loss-gradient phase below
    constexpr int HB_PRE = 4;
    uint4 pre[HB_PRE];
#pragma unroll
    for (int k = 0; k < HB_PRE; ++k) {
        const int r = r0 + grp + k * HB_GROUPS;
        if (r < r1) pre[k] = ld_last_use(H2 + (size_t)r * kH + j0);
    }
    for (int i = threadIdx.x; i < r1 - r0; i += blockDim.x) {  // each row's loss gradient once
        float gr, se;
        if (zpart) head_row(zpart, zparts, y, b3, B, r0 + i, gr, se);
        else gr = g3[r0 + i], se = sqerr[r0 + i];
        sg[i] = gr;
        ss[i] = se;
    }
    __syncthreads();
    // one row: dZ2 = g3 * w3 where H2 > 0, and the running sums
    auto row = [&](int r, const uint4& raw) {
        const float gr = sg[r - r0], se = ss[r - r0];
        float h[8];
        const __nv_bfloat162* hb = reinterpret_cast<const __nv_bfloat162*>(&raw);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float2 x = __bfloat1622float2(hb[e]);
            h[2 * e] = x.x;
            h[2 * e + 1] = x.y;
        }
        __align__(16) __nv_bfloat162 d[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float d0 = h[2 * e] > 0.f ? gr * w[2 * e] : 0.f, d1 = h[2 * e + 1] > 0.f ? gr * w[2 * e + 1] : 0.f;
            d[e] = __floats2bfloat162_rn(d0, d1);
            ab[2 * e] += d0;
            ab[2 * e + 1] += d1;
            aw[2 * e] = fmaf(gr, h[2 * e], aw[2 * e]);
            aw[2 * e + 1] = fmaf(gr, h[2 * e + 1], aw[2 * e + 1]);
        }
        *reinterpret_cast<uint4*>(dZ2 + (size_t)r * kH + j0) = *reinterpret_cast<const uint4*>(d);
        if (first) {
            ag += gr;
            al += se;
        }
    };
#pragma unroll
    for (int k = 0; k < HB_PRE; ++k) {
        const int r = r0 + grp + k * HB_GROUPS;
        if (r < r1) row(r, pre[k]);
    }
#pragma unroll 4
    for (int r = r0 + grp + HB_PRE * HB_GROUPS; r < r1; r += HB_GROUPS)
        row(r, ld_last_use(H2 + (size_t)r * kH + j0));
    if (grp > 0) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            sh[grp - 1][j0 + e] = ab[e];
            sh[grp - 1][kH + j0 + e] = aw[e];
        }
        if (first) {
            sh[grp - 1][2 * kH] = ag;
            sh[grp - 1][2 * kH + 1] = al;
        }
    }
    __syncthreads();
    if (grp == 0) {
        float* out = part + (size_t)blockIdx.x * HB_COLS;
        for (int g = 0; g < HB_GROUPS - 1; ++g) {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                ab[e] += sh[g][j0 + e];
                aw[e] += sh[g][kH + j0 + e];
            }
            if (first) {
                ag += sh[g][2 * kH];
                al += sh[g][2 * kH + 1];
            }
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            out[j0 + e] = ab[e];
            out[kH + j0 + e] = aw[e];
        }
        if (first) {
            out[2 * kH] = ag;
            out[2 * kH + 1] = al;
        }
    }
}

// the chunk's column sums of a [B][kH] BF16 matrix into row blockIdx.x of
// part[chunks][kH] (db1 = sum_b dZ1)
__global__ void __launch_bounds__(256) colsum_kernel(const __nv_bfloat16* X, int B, float* part) {
    __shared__ float sh[HB_GROUPS - 1][kH];
    const int grp = threadIdx.x >> 6, j0 = (threadIdx.x & 63) * 8;
    float a[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) a[e] = 0.f;
    const int r0 = blockIdx.x * HB_ROWS, r1 = min(r0 + HB_ROWS, B);
#pragma unroll 4
    for (int r = r0 + grp; r < r1; r += HB_GROUPS) {
        float v[8];
        load8(X + (size_t)r * kH + j0, v);
#pragma unroll
        for (int e = 0; e < 8; ++e) a[e] += v[e];
    }
    if (grp > 0)
#pragma unroll
        for (int e = 0; e < 8; ++e) sh[grp - 1][j0 + e] = a[e];
    __syncthreads();
    if (grp == 0) {
        for (int g = 0; g < HB_GROUPS - 1; ++g)
#pragma unroll
            for (int e = 0; e < 8; ++e) a[e] += sh[g][j0 + e];
#pragma unroll
        for (int e = 0; e < 8; ++e) part[(size_t)blockIdx.x * kH + j0 + e] = a[e];
    }
}

// Adam (Kingma & Ba, Algorithm 1) on the flat FP32 parameters, then the BF16
// copies the GEMMs read.  bc1 = 1 - beta1^t, bc2 = 1 - beta2^t.
// The updated weights also go to their BF16 copies: W1 | W2 | w3 back to
// back in bf, the flat vector's layout W1 | b1 | W2 | b2 | w3 | b3 without
// the biases (each bias is kH long; b3 is last).
struct BfCopy {
    __nv_bfloat16* bf;
    long long ob1, oW2, ob2, ow3, ob3;
};

// The backward pass's last launch: each parameter's gradient from the
// partial sums the earlier kernels left, then either the gradient stored
// in g (adam == 0) or one Adam step applied in place (p, m, v and the BF16
// copies).  Partials:
//   w1p [s1][kH * kpad], w2p [s2][kH * kH]  split-K sums of dW1, dW2;
//   cp  [crows][kH]                         row-group sums of db1;
//   hp  [hrows][HB_COLS]                    row-chunk sums of db2 | dw3 |
//                                           db3 | squared error.
// The first FIN_LONG blocks take 32 columns each of cp, then of hp: their
// warps stride down the rows (lane = column) and the warp sums are added in
// a fixed order; the nwide blocks after them take W1 and W2, four elements
// per thread, adding the splits in order.  The loss is the squared-error
// column / B.
struct FinishArgs {
    const float *w1p, *w2p, *cp, *hp;
    int s1, s2, crows, hrows;
    long long n1, n2;  // kH * kpad, kH * kH
    int nwide;
    float* g;
    float *p, *m, *v;
    float lr, bc1, bc2;
    BfCopy c;
    float* loss;
    float inv_b;
    int adam;
};

__device__ __forceinline__ void apply_grad(const FinishArgs& a, long long i, float gi) {
    if (!a.adam) {
        a.g[i] = gi;
        return;
    }
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float mi = b1 * a.m[i] + (1.f - b1) * gi;
    const float vi = b2 * a.v[i] + (1.f - b2) * gi * gi;
    a.m[i] = mi;
    a.v[i] = vi;
    const float pi = a.p[i] - a.lr * (mi / a.bc1) / (sqrtf(vi / a.bc2) + eps);
    a.p[i] = pi;
    const BfCopy& c = a.c;
    if (i < c.ob1) c.bf[i] = __float2bfloat16_rn(pi);
    else if (i >= c.oW2 && i < c.ob2) c.bf[i - kH] = __float2bfloat16_rn(pi);
    else if (i >= c.ow3 && i < c.ob3) c.bf[i - 2 * kH] = __float2bfloat16_rn(pi);
}

// the same for four consecutive weights (i a multiple of 4, inside W1 or
// W2), with their Adam state m0, v0, p0 read before the gradient was formed
__device__ __forceinline__ void adam4(const FinishArgs& a, long long i, const float4& g, const float4& m0,
                                      const float4& v0, const float4& p0) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float gs[4] = {g.x, g.y, g.z, g.w}, ms[4] = {m0.x, m0.y, m0.z, m0.w}, vs[4] = {v0.x, v0.y, v0.z, v0.w},
                ps[4] = {p0.x, p0.y, p0.z, p0.w};
    float mo[4], vo[4], po[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        mo[k] = b1 * ms[k] + (1.f - b1) * gs[k];
        vo[k] = b2 * vs[k] + (1.f - b2) * gs[k] * gs[k];
        po[k] = ps[k] - a.lr * (mo[k] / a.bc1) / (sqrtf(vo[k] / a.bc2) + eps);
    }
    *reinterpret_cast<float4*>(a.m + i) = make_float4(mo[0], mo[1], mo[2], mo[3]);
    *reinterpret_cast<float4*>(a.v + i) = make_float4(vo[0], vo[1], vo[2], vo[3]);
    *reinterpret_cast<float4*>(a.p + i) = make_float4(po[0], po[1], po[2], po[3]);
    const long long j = i < a.c.ob1 ? i : i - kH;  // W1 | W2 back to back in the BF16 copy
    __align__(8) __nv_bfloat162 h[2] = {__floats2bfloat162_rn(po[0], po[1]), __floats2bfloat162_rn(po[2], po[3])};
    *reinterpret_cast<uint2*>(a.c.bf + j) = *reinterpret_cast<const uint2*>(h);
}

constexpr int FIN_THREADS = 256, FIN_WARPS = FIN_THREADS / 32, FIN_BATCH = 10, FIN_ROWS = 16;
constexpr int FIN_LONG = kH / 32 + (HB_COLS + 31) / 32;  // blocks of 32 bias / head columns

// at most 85 registers a thread: three 256-thread blocks per SM, so the 433
// blocks of a 65,536-row step (W1 and W2 four weights a thread, plus the bias
// columns) run in one wave on 148 SMs
__global__ void __launch_bounds__(FIN_THREADS, 3) finish_kernel(FinishArgs a) {
    pdl_wait();
    if ((int)blockIdx.x >= FIN_LONG) {  // W1 and W2: four elements per thread, FIN_BATCH splits in flight
        const long long t = (long long)(blockIdx.x - FIN_LONG) * FIN_THREADS + threadIdx.x, e = 4 * t;
        if (e >= a.n1 + a.n2) return;
        const bool w1 = e < a.n1;
        const float* src = w1 ? a.w1p + e : a.w2p + (e - a.n1);
        const long long stride = w1 ? a.n1 : a.n2, flat = w1 ? e : a.c.oW2 + (e - a.n1);
        const int splits = w1 ? a.s1 : a.s2;
        float4 m0, v0, p0;  // the Adam state, fetched while the partials are
        if (a.adam) {
            m0 = *reinterpret_cast<const float4*>(a.m + flat);
            v0 = *reinterpret_cast<const float4*>(a.v + flat);
            p0 = *reinterpret_cast<const float4*>(a.p + flat);
        }
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        // every batch issues all its loads (those past the last split are
        // predicated off) before adding them in split order, so a split count
        // that is not a multiple of the batch costs no extra round trips
        for (int s0 = 0; s0 < splits; s0 += FIN_BATCH) {
            float4 x[FIN_BATCH];
#pragma unroll
            for (int k = 0; k < FIN_BATCH; ++k)
                if (s0 + k < splits) x[k] = __ldcg(reinterpret_cast<const float4*>(src + (size_t)(s0 + k) * stride));
#pragma unroll
            for (int k = 0; k < FIN_BATCH; ++k) {
                if (s0 + k < splits) {
                    acc.x += x[k].x;
                    acc.y += x[k].y;
                    acc.z += x[k].z;
                    acc.w += x[k].w;
                }
            }
        }
        if (a.adam) {
            adam4(a, flat, acc, m0, v0, p0);
        } else {
            a.g[flat] = acc.x;
            a.g[flat + 1] = acc.y;
            a.g[flat + 2] = acc.z;
            a.g[flat + 3] = acc.w;
        }
        return;
    }
    // 32 columns of the db1 row-group sums, then of the head's chunk sums: the
    // warps stride down the rows (lane = column), eight rows in flight each
    __shared__ float sh[FIN_WARPS][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int blk = (int)blockIdx.x;
    const bool bias1 = blk < kH / 32;
    if (!bias1) blk -= kH / 32;
    const int col = blk * 32 + lane, ncols = bias1 ? kH : HB_COLS, rows = bias1 ? a.crows : a.hrows;
    const float* src = bias1 ? a.cp : a.hp;
    float x = 0.f;
    if (col < ncols) {  // FIN_ROWS rows of a warp in flight, added in row order
        for (int r0 = w; r0 < rows; r0 += FIN_WARPS * FIN_ROWS) {
            float v[FIN_ROWS];
#pragma unroll
            for (int k = 0; k < FIN_ROWS; ++k)
                if (r0 + k * FIN_WARPS < rows) v[k] = __ldcg(src + (size_t)(r0 + k * FIN_WARPS) * ncols + col);
#pragma unroll
            for (int k = 0; k < FIN_ROWS; ++k)
                if (r0 + k * FIN_WARPS < rows) x += v[k];
        }
    }
    sh[w][lane] = x;
    __syncthreads();
    if (w != 0 || col >= ncols) return;
    float t = 0.f;
    for (int k = 0; k < FIN_WARPS; ++k) t += sh[k][lane];
    if (bias1) apply_grad(a, a.c.ob1 + col, t);
    else if (col < kH) apply_grad(a, a.c.ob2 + col, t);
    else if (col < 2 * kH) apply_grad(a, a.c.ow3 + (col - kH), t);
    else if (col == 2 * kH) apply_grad(a, a.c.ob3, t);
    else if (a.loss) a.loss[0] = t * a.inv_b;
}

__global__ void to_bf16_kernel(const float* src, __nv_bfloat16* dst, long long n) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __float2bfloat16_rn(src[i]);
}

// ---------------------------------------------------------- env -> input --
// Row of the net input for a position: bf16 1.0 at column c for each P1 stone
// on cell c, at column cells + c for each P2 stone, at column 2*cells when P1
// is to move; zero elsewhere up to ld.
template <class G>
__device__ __forceinline__ void write_input_row(const G& g, __nv_bfloat16* row, int ld) {
    const __nv_bfloat16 one = __float2bfloat16_rn(1.f), zero = __float2bfloat16_rn(0.f);
    const int cells = cells_of(g);
    for (int c0 = 0; c0 < ld; c0 += 8) {
        __align__(16) __nv_bfloat16 v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            int c = c0 + i;
            bool on = false;
            if (c < cells) {
                int b = g.bit_of(c);
                on = g.side == 0 ? mask_has(g.own, b) : mask_has(g.opp, b);
            } else if (c < 2 * cells) {
                int b = g.bit_of(c - cells);
                on = g.side == 0 ? mask_has(g.opp, b) : mask_has(g.own, b);
            } else if (c == 2 * cells) {
                on = g.side == 0;
            }
            v[i] = on ? one : zero;
        }
        *reinterpret_cast<uint4*>(row + c0) = *reinterpret_cast<const uint4*>(v);
    }
}

template <class G>
__global__ void pack_inputs_kernel(EnvDev d, __nv_bfloat16* X, int ld) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= d.n) return;
    G g;
    set_table(g, nullptr);
    load_state(g, d, e);
    write_input_row(g, X + (size_t)e * ld, ld);
}

// The same input row as bits (bit c = column c) in four words: P1's stones
// in canonical cell order, then P2's shifted up by `cells`, then the
// P1-to-move bit at 2 * cells (at most 255 columns).
template <class G>
__device__ __forceinline__ void input_bits(const G& g, uint64_t x[4]) {
    const int cells = cells_of(g);
    const typename G::Mask& p1 = g.side == 0 ? g.own : g.opp;
    const typename G::Mask& p2 = g.side == 0 ? g.opp : g.own;
    const uint64_t a0 = canon_mask_word(g, p1, 0), a1 = cells > 64 ? canon_mask_word(g, p1, 1) : 0ull;
    const uint64_t b0 = canon_mask_word(g, p2, 0), b1 = cells > 64 ? canon_mask_word(g, p2, 1) : 0ull;
    const uint32_t r = (uint32_t)cells & 63u;  // P2 starts in word cells / 64 (0 or 1) at bit r
    const uint64_t lo = shl64c(b0, r), mid = shl64c(b1, r) | shr64c(b0, 64u - r), hi = shr64c(b1, 64u - r);
    const bool up = cells >= 64;
    x[0] = a0 | (up ? 0ull : lo);
    x[1] = a1 | (up ? lo : mid);
    x[2] = up ? mid : hi;
    x[3] = up ? hi : 0ull;
    const int s = 2 * cells;
    const uint64_t side_bit = g.side == 0 ? (1ull << (s & 63)) : 0ull;
#pragma unroll
    for (int w = 0; w < 4; ++w) x[w] |= (s >> 6) == w ? side_bit : 0ull;  // no run-time index into x
}

// bits t0, t0+1 of v as two BF16 values (1.0 = 0x3F80) in one 32-bit word
__device__ __forceinline__ uint32_t bf16_pair(uint32_t v) { return ((v & 1u) | ((v & 2u) << 15)) * 0x3F80u; }

// Continuation j of env e0+i (i < n_chunk): up to `plies` uniform-random plies
// from the stored state with the draws of playout seed + j, then either the
// final result (score, done = 1) or the leaf's input row (done = 0).  The rows
// are written by the whole warp together: each lane's bits go to shared memory,
// then row by row every lane expands one byte (8 columns) into one 16-byte
// store, so a row is one contiguous write.  Only the first kuse columns are
// written (the layer that reads them takes no more).
constexpr int LEAF_THREADS = 128;
template <class G>
__global__ void __launch_bounds__(LEAF_THREADS) leaf_kernel(EnvDev d, long long e0, long long n_chunk, int K,
                                                             uint64_t seed, int plies, __nv_bfloat16* X, int ld,
                                                             int kuse, float* score, uint8_t* done, long long rows_pad) {
    pdl_wait();
    __shared__ uint64_t bits[LEAF_THREADS / 32][32][4];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x, total = n_chunk * K;
    uint64_t x[4] = {0ull, 0ull, 0ull, 0ull};
    if (t < total) {
        const long long e = e0 + t / K;
        const int j = (int)(t % K);
        G g;
        set_table(g, nullptr);
        load_state(g, d, e);
        uint64_t key = env_key(splitmix64(seed + (uint64_t)j), (uint64_t)(d.env_offset + e));
        int stop = g.ply + plies;
        uint32_t rhi = draw_hi(key, (uint32_t)g.ply);
        while (g.outcome == kOngoing && g.ply < stop) random_ply_pre(g, key, rhi);
        if (g.outcome != kOngoing) {
            score[t] = p1_score(g.outcome);
            done[t] = 1;
        } else {
            done[t] = 0;
        }
        input_bits(g, x);
    }
#pragma unroll
    for (int w = 0; w < 4; ++w) bits[wib][lane][w] = x[w];
    __syncwarp();
    const long long t0 = t - lane;
    const uint8_t* rb = reinterpret_cast<const uint8_t*>(&bits[wib][0][0]);
    if (8 * lane < kuse) {
        for (int r = 0; r < 32 && t0 + r < rows_pad; ++r) {  // rows past the last continuation: zero
            const uint32_t v = rb[r * 32 + lane];  // columns 8 * lane .. 8 * lane + 7 of row t0 + r
            const uint4 o = make_uint4(bf16_pair(v), bf16_pair(v >> 2), bf16_pair(v >> 4), bf16_pair(v >> 6));
            *reinterpret_cast<uint4*>(X + (size_t)(t0 + r) * ld + 8 * lane) = o;
        }
    }
}

// value[e0+i] = mean over j of (done ? score : p_net)
__global__ void combine_kernel(long long e0, long long n_chunk, int K, const float* score, const uint8_t* done,
                               const float* p, float* value) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_chunk) return;
    float a = 0.f;
    for (int j = 0; j < K; ++j) {
        long long t = i * K + j;
        a += done[t] ? score[t] : p[t];
    }
    value[e0 + i] = a / (float)K;
}

// The same mean with each continuation's p formed here from its row's head
// partials (as head_finish_kernel forms it): one launch instead of two.
__global__ void combine_z_kernel(long long e0, long long n_chunk, int K, const float* score, const uint8_t* done,
                                 const float* zpart, int parts, const float* b3, float* value) {
    pdl_wait();
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_chunk) return;
    float a = 0.f;
    for (int j = 0; j < K; ++j) {
        long long t = i * K + j;
        if (done[t]) {
            a += score[t];
        } else {
            float z = 0.f;
            for (int q = 0; q < parts; ++q) z += zpart[(size_t)t * parts + q];
            const float v = tanhf(z + b3[0]);
            a += 0.5f * (v + 1.f);
        }
    }
    value[e0 + i] = a / (float)K;
}

unsigned blocks_for(long long n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

struct ludax_net {
    int cells, kin, kpad;
    int use_tcgen05;  // forward layers on tcgen05 (1, default; 2: never the one-launch MLP) or mma.sync (0)
    long long max_batch;
    cudaStream_t stream;
    long long nparams;
    long long oW1, ob1, oW2, ob2, ow3, ob3;
    int t;  // Adam steps taken
    float *p, *m, *v, *g;
    __nv_bfloat16 *W1b, *W2b, *w3b;
    __nv_bfloat16 *H1, *H2, *dZ2, *dZ1, *Xleaf;
    uint32_t* h1bits;  // which values of H1 are non-zero (h1bits_index layout), from the one-launch training forward
    bool h1bits_set;   // the last training forward wrote h1bits
    float *pout, *g3, *sqerr, *score;
    // backward partial sums (see finish_kernel): the training forward's head
    // partials [B][ZPARTS], the head's row-chunk sums, db1's row-group sums
    // and the split-K sums of dW2 and dW1
    float *zp, *hp, *cp, *w2p, *w1p;
    long long cp_rows, w2_floats, w1_floats;
    int zparts;  // head partials per row the last training forward left in zp
    uint8_t* done;
    __nv_bfloat16* mlp_scratch;  // layer-1 rows of the fused inference kernel (allocated on first use)
    float* mlp_z;                // its head partials, 4 per row
    int mlp_rows;
};

namespace {

int net_check(const ludax_net* n, long long B) {
    if (!n || B < 1 || B > n->max_batch) return LUDAX_ERR_ARG;
    if (B % BM) return LUDAX_ERR_SIZE;
    return LUDAX_OK;
}

int refresh_bf16(ludax_net* n) {
    to_bf16_kernel<<<blocks_for((long long)kH * n->kpad, 256), 256, 0, n->stream>>>(n->p + n->oW1, n->W1b,
                                                                                   (long long)kH * n->kpad);
    to_bf16_kernel<<<blocks_for((long long)kH * kH, 256), 256, 0, n->stream>>>(n->p + n->oW2, n->W2b, (long long)kH * kH);
    to_bf16_kernel<<<blocks_for(kH, 256), 256, 0, n->stream>>>(n->p + n->ow3, n->w3b, kH);
    return cudaGetLastError() == cudaSuccess ? LUDAX_OK : LUDAX_ERR_CUDA;
}

// One hidden layer out = bf16(relu(A . W^T + b)): on the tcgen05 tensor
// cores (TMA + TMEM) when the shape allows, else the mma.sync kernel.
int dense_layer(ludax_net* n, const __nv_bfloat16* A, const __nv_bfloat16* W, const float* b, __nv_bfloat16* out,
                long long B, int K) {
    if (n->use_tcgen05 && umma_dense_supported((int)B, kH, K))
        return umma_dense_relu(A, W, b, out, (int)B, kH, K, kH, n->stream);
    GemmArgs a{};
    a.A = A; a.B = W; a.M = (int)B; a.N = kH; a.K = K; a.lda = K; a.ldb = K; a.bias = b; a.out = out; a.ldo = kH;
    return launch_gemm<true, true, EPI_BIAS_RELU>(a, 1, n->stream);
}

// p[row] from the head partials of the fused second layer; with labels also
// g3[row] = dL/dz for L = mean (p - y)^2 and the row's squared error
__global__ void head_finish_kernel(const float* zpart, int parts, const float* b3, int B, float* p_out,
                                   const float* y, float* g3, float* sqerr) {
    int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= B) return;
    float z = 0.f;
    for (int i = 0; i < parts; ++i) z += zpart[(size_t)row * parts + i];
    const float v = tanhf(z + b3[0]), p = 0.5f * (v + 1.f);
    if (p_out) p_out[row] = p;
    if (y) {
        const float d = p - y[row];
        g3[row] = d * (1.f - v * v) / (float)B;  // 2 (p-y)/B * (1/2) (1 - v^2)
        sqerr[row] = d * d;
    }
}

// Training runs both hidden layers and the backward contractions on
// tcgen05 for these batches; otherwise on the mma.sync kernel.
bool tc_layers(const ludax_net* n, long long B) {
    return n->use_tcgen05 && umma_dense_supported((int)B, kH, kH);
}

// Inference runs on tcgen05 (the layers, with the head in the second one's
// epilogue) for these batches and input widths.
bool infer_tc(const ludax_net* n, long long B, int kuse) {
    return n->use_tcgen05 && umma_dense_supported((int)B, kH, kuse) && umma_dense_supported((int)B, kH, kH);
}

// Both hidden layers and the head's dot products of an inference forward (no
// labels): the partials of each row's z into *zpart, *parts per row -- from
// the one-launch MLP (layer 1's rows through an L2-resident scratch), or from
// two layer launches when the scratch cannot be had or tensor path 2 is set.
int infer_head(ludax_net* n, const __nv_bfloat16* X, long long B, int kuse, const float** zpart_out, int* parts_out) {
    cudaStream_t s = n->stream;
    if (!n->mlp_scratch && n->use_tcgen05 == 1) {
        const int rows = umma_mlp_scratch_rows();
        if (rows > 0 && cudaMalloc(&n->mlp_scratch, sizeof(__nv_bfloat16) * (size_t)rows * kH) == cudaSuccess &&
            cudaMalloc(&n->mlp_z, sizeof(float) * 4 * (size_t)n->max_batch) == cudaSuccess) {
            n->mlp_rows = rows;
        } else {  // no scratch: the two-launch form below
            cudaGetLastError();
            cudaFree(n->mlp_scratch);
            n->mlp_scratch = nullptr;
        }
    }
    int st;
    float* zpart;
    if (n->mlp_scratch && n->use_tcgen05 == 1) {  // both layers and the head in one launch, layer 1's rows through L2
        zpart = n->mlp_z;
        *parts_out = 4;
        st = umma_mlp_head(X, n->kpad, kuse, n->W1b, n->kpad, n->p + n->ob1, n->W2b, n->p + n->ob2, n->w3b, zpart,
                           n->mlp_scratch, n->mlp_rows, (int)B, s);
    } else {
        zpart = n->g3;  // 2 floats per row: g3 and sqerr are unused without labels
        *parts_out = kH / 256;
        st = umma_dense_relu_ex(X, n->kpad, n->W1b, n->kpad, n->p + n->ob1, n->H1, kH, nullptr, nullptr, (int)B, kH,
                                kuse, s);
        if (!st)
            st = umma_dense_relu_ex(n->H1, kH, n->W2b, kH, n->p + n->ob2, nullptr, 0, n->w3b, zpart, (int)B, kH, kH, s);
    }
    *zpart_out = zpart;
    return st;
}

// Forward pass to p (and, with labels y, the per-row gradient g3 of the loss,
// or on the tcgen05 training path the head partials it is formed from; p is
// then not written).
// kuse <= kpad: the input columns the first layer reads (the rest must be zero).
// Without labels (inference) and on the tcgen05 path, the head is fused into
// the second layer's epilogue, so its rows are never stored.
int net_forward(ludax_net* n, const __nv_bfloat16* X, long long B, float* p, const float* y, int kuse = 0) {
    cudaStream_t s = n->stream;
    if (kuse <= 0) kuse = n->kpad;
    if (!y && p && infer_tc(n, B, kuse)) {
        const float* zpart;
        int parts;
        const int st = infer_head(n, X, B, kuse, &zpart, &parts);
        if (st) return st;
        head_finish_kernel<<<blocks_for(B, 256), 256, 0, s>>>(zpart, parts, n->p + n->ob3, (int)B, p, nullptr,
                                                               nullptr, nullptr);
        return cudaGetLastError() == cudaSuccess ? LUDAX_OK : LUDAX_ERR_CUDA;
    }
    int st;
    if (tc_layers(n, B)) {
        // training forward: both layers in one launch (layer 1's rows pass
        // through L2 on their way to layer 2 and are kept, as are layer 2's;
        // tensor path 2 keeps two launches);
        // layer 1 reads the input columns up to the next multiple of 64 past
        // the last used one (the rest are zero by the input contract); the
        // head's dot products come out as four partials per row, from which
        // the backward pass's first kernel forms the loss gradient
        const int k1 = std::min(n->kpad, (n->kin + 63) / 64 * 64);
        n->h1bits_set = n->use_tcgen05 == 1;
        if (n->use_tcgen05 == 1) {
            n->zparts = ZPARTS;
            return umma_mlp_train(X, n->kpad, k1, n->W1b, n->kpad, n->p + n->ob1, n->W2b, n->p + n->ob2, n->w3b,
                                  n->zp, n->H1, n->H2, n->h1bits, (int)B, s);
        }
        // the two-launch form (tensor path 2): the second layer's epilogue takes two head partials per row
        n->zparts = kH / 256;
        if ((st = umma_dense_relu_ex(X, n->kpad, n->W1b, n->kpad, n->p + n->ob1, n->H1, kH, nullptr, nullptr, (int)B,
                                     kH, k1, s)))
            return st;
        return umma_dense_relu_ex(n->H1, kH, n->W2b, kH, n->p + n->ob2, n->H2, kH, n->w3b, n->zp, (int)B, kH, kH, s);
    }
    n->h1bits_set = false;
    if ((st = dense_layer(n, X, n->W1b, n->p + n->ob1, n->H1, B, n->kpad))) return st;
    if ((st = dense_layer(n, n->H1, n->W2b, n->p + n->ob2, n->H2, B, kH))) return st;
    head_forward_kernel<<<blocks_for(B, 8), 256, 0, s>>>(n->H2, n->w3b, n->p + n->ob3, (int)B, p, y, n->g3, n->sqerr);
    return cudaGetLastError() == cudaSuccess ? LUDAX_OK : LUDAX_ERR_CUDA;
}

struct AdamStep {
    float lr, bc1, bc2;
};

// Backward pass after net_forward with labels y: the gradient into n->g
// (adam == nullptr) or one Adam step applied to the parameters, and the mean
// loss into loss_out (nullable).  Launches: the head's backward (dZ2 and its
// bias / weight sums), dW2 as split-K partials, dZ1 with db1's column sums,
// dW1 as split-K partials, and finish_kernel, which reduces every partial and
// stores or applies the gradient.
int net_backward(ludax_net* n, const __nv_bfloat16* X, long long B, const float* y, float* loss_out,
                 const AdamStep* adam) {
    cudaStream_t s = n->stream;
    const int chunks = (int)((B + HB_ROWS - 1) / HB_ROWS);
    const bool tc = tc_layers(n, B);
    if (launch_dependent(head_backward_kernel, (unsigned)chunks, 256, 0, s, (const __nv_bfloat16*)n->H2,
                         (const __nv_bfloat16*)n->w3b, (const float*)n->g3, (const float*)n->sqerr,
                         (const float*)(tc ? n->zp : nullptr), n->zparts, y, (const float*)(n->p + n->ob3), (int)B, n->dZ2,
                         n->hp) != cudaSuccess)
        return LUDAX_ERR_CUDA;
    // dW2 = dZ2^T . H1 and dW1 = dZ1^T . X, split over the batch into partial sums.
    // dW2 runs first, while the dZ2 rows just written are still in L2; dZ1
    // then runs just before dW1, which reads the dZ1 rows it leaves in L2.
    auto weight_grad = [&](const __nv_bfloat16* A, const __nv_bfloat16* Bm, int N, int ldb, float* part,
                           long long cap, int& splits, int last_use) -> int {
        if (tc && umma_dense_supported(kH, N, (int)B))
            return umma_grad_weights(A, kH, Bm, ldb, kH, N, (int)B, part, cap, &splits, s, last_use);
        splits = (int)std::min<long long>(32, B / BKT);
        while (splits > 1 && (B % ((long long)BKT * splits))) --splits;
        GemmArgs a{};
        a.A = A; a.B = Bm; a.M = kH; a.N = N; a.K = (int)B; a.lda = kH; a.ldb = ldb; a.partial = part;
        return launch_gemm<false, false, EPI_PARTIAL>(a, splits, s);
    };
    int st, s2 = 0, s1 = 0;
    // dW2's last use is of H1 (dZ2 is read again by dZ1), dW1's of dZ1
    if ((st = weight_grad(n->dZ2, n->H1, kH, kH, n->w2p, n->w2_floats, s2, 2))) return st;
    // dZ1 = (dZ2 . W2) * [H1 > 0], and db1 = its column sums as partial rows
    int crows;
    if (tc) {
        crows = umma_grad_colrows((int)B, kH);
        if (crows <= 0 || crows > n->cp_rows) return LUDAX_ERR_CUDA;
        // the mask from H1's bits when the forward left them (4 MB instead of H1's 64 MB at 65,536 rows)
        st = n->h1bits_set ? umma_grad_maskbits(n->dZ2, n->W2b, n->h1bits, n->dZ1, (int)B, kH, kH, n->cp, s)
                           : umma_grad_mask(n->dZ2, n->W2b, n->H1, n->dZ1, (int)B, kH, kH, n->cp, s);
    } else {
        GemmArgs a{};
        a.A = n->dZ2; a.B = n->W2b; a.M = (int)B; a.N = kH; a.K = kH; a.lda = kH; a.ldb = kH;
        a.mask = n->H1; a.out = n->dZ1; a.ldo = kH;
        st = launch_gemm<true, false, EPI_MASK>(a, 1, s);
        if (!st) colsum_kernel<<<chunks, 256, 0, s>>>(n->dZ1, (int)B, n->cp);
        crows = chunks;
    }
    if (st) return st;
    if ((st = weight_grad(n->dZ1, X, n->kpad, n->kpad, n->w1p, n->w1_floats, s1, 1))) return st;
    FinishArgs f{};
    f.w1p = n->w1p; f.w2p = n->w2p; f.cp = n->cp; f.hp = n->hp;
    f.s1 = s1; f.s2 = s2; f.crows = crows; f.hrows = chunks;
    f.n1 = (long long)kH * n->kpad; f.n2 = (long long)kH * kH;
    f.nwide = (int)blocks_for((f.n1 + f.n2) / 4, FIN_THREADS);
    f.g = n->g; f.p = n->p; f.m = n->m; f.v = n->v;
    if (adam) {
        f.adam = 1;
        f.lr = adam->lr; f.bc1 = adam->bc1; f.bc2 = adam->bc2;
    }
    f.c = BfCopy{n->W1b, n->ob1, n->oW2, n->ob2, n->ow3, n->ob3};
    f.loss = loss_out;
    f.inv_b = 1.f / (float)B;
    return launch_dependent(finish_kernel, (unsigned)(FIN_LONG + f.nwide), FIN_THREADS, 0, s, f) ==
                   cudaSuccess
               ? LUDAX_OK
               : LUDAX_ERR_CUDA;
}

}  // namespace

extern "C" {

int ludax_net_create(ludax_net** out, int32_t cells, int64_t max_batch, void* stream) {
    if (!out || cells < 1 || cells > 127 || max_batch < BM || max_batch % BM || max_batch > (1ll << 24))
        return LUDAX_ERR_ARG;
    *out = nullptr;
    ludax_net* n = new (std::nothrow) ludax_net();
    if (!n) return LUDAX_ERR_NOMEM;
    n->cells = cells;
    n->kin = 2 * cells + 1;
    n->kpad = ((n->kin + 127) / 128) * 128;
    n->max_batch = max_batch;
    n->stream = (cudaStream_t)stream;
    n->use_tcgen05 = 1;
    n->oW1 = 0;
    n->ob1 = n->oW1 + (long long)kH * n->kpad;
    n->oW2 = n->ob1 + kH;
    n->ob2 = n->oW2 + (long long)kH * kH;
    n->ow3 = n->ob2 + kH;
    n->ob3 = n->ow3 + kH;
    n->nparams = n->ob3 + 1;
    const long long B = max_batch;
    const int max_splits = 48, sms = device_sms();  // split-K partials: the SM count over the tiles (37 for dW1 on 148 SMs)
    if (sms <= 0) {
        delete n;
        return LUDAX_ERR_CUDA;
    }
    const long long chunks = (B + HB_ROWS - 1) / HB_ROWS;
    auto up4 = [](long long x) { return (x + 3) / 4 * 4; };  // regions start 16-byte aligned
    n->cp_rows = std::max<long long>(chunks, 4ll * sms);      // colsum_kernel's chunks or the tcgen05 row groups
    n->w2_floats = (long long)max_splits * kH * kH;
    n->w1_floats = (long long)max_splits * kH * n->kpad;
    const long long zp_f = ZPARTS * B, hp_f = up4(chunks * HB_COLS), cp_f = n->cp_rows * kH;
    const long long part_floats = zp_f + hp_f + cp_f + n->w2_floats + n->w1_floats;
    // p, m, v and g each start on a 16-byte boundary (the finish kernel
    // reads and writes the Adam state four weights at a time)
    const long long pstride = up4(n->nparams);
    bool ok = cudaMalloc(&n->p, 4 * pstride * sizeof(float)) == cudaSuccess;
    if (ok) {
        n->m = n->p + pstride;
        n->v = n->m + pstride;
        n->g = n->v + pstride;
    }
    ok = ok && cudaMalloc(&n->W1b, sizeof(__nv_bfloat16) * ((size_t)kH * n->kpad + (size_t)kH * kH + kH)) == cudaSuccess;
    if (ok) {
        n->W2b = n->W1b + (size_t)kH * n->kpad;
        n->w3b = n->W2b + (size_t)kH * kH;
    }
    // H1 | H2 | dZ2 | dZ1 | Xleaf, then H1's bit mask (kH / 32 words per row)
    ok = ok && cudaMalloc(&n->H1, sizeof(__nv_bfloat16) * (size_t)B * (4 * kH + n->kpad + kH / 16)) == cudaSuccess;
    if (ok) {
        n->H2 = n->H1 + (size_t)B * kH;
        n->dZ2 = n->H2 + (size_t)B * kH;
        n->dZ1 = n->dZ2 + (size_t)B * kH;
        n->Xleaf = n->dZ1 + (size_t)B * kH;
        n->h1bits = reinterpret_cast<uint32_t*>(n->Xleaf + (size_t)B * n->kpad);
    }
    ok = ok && cudaMalloc(&n->pout, sizeof(float) * (4 * (size_t)B + part_floats)) == cudaSuccess;
    if (ok) {
        n->g3 = n->pout + B;
        n->sqerr = n->g3 + B;
        n->score = n->sqerr + B;
        n->zp = n->score + B;
        n->hp = n->zp + zp_f;
        n->cp = n->hp + hp_f;
        n->w2p = n->cp + cp_f;
        n->w1p = n->w2p + n->w2_floats;
    }
    ok = ok && cudaMalloc(&n->done, (size_t)B) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        ludax_net_destroy(n);
        return LUDAX_ERR_NOMEM;
    }
    if (cudaMemsetAsync(n->p, 0, 4 * (size_t)(n->m - n->p) * sizeof(float), n->stream) != cudaSuccess ||
        refresh_bf16(n) != LUDAX_OK) {
        ludax_net_destroy(n);
        return LUDAX_ERR_CUDA;
    }
    *out = n;
    return LUDAX_OK;
}

int ludax_net_destroy(ludax_net* n) {
    if (!n) return LUDAX_OK;
    cudaStreamSynchronize(n->stream);
    cudaFree(n->p);
    cudaFree(n->W1b);
    cudaFree(n->H1);
    cudaFree(n->pout);
    cudaFree(n->done);
    if (n->mlp_scratch) cudaFree(n->mlp_scratch);
    if (n->mlp_z) cudaFree(n->mlp_z);
    delete n;
    return cudaGetLastError() == cudaSuccess ? LUDAX_OK : LUDAX_ERR_CUDA;
}

int ludax_net_sizes(const ludax_net* n, int32_t* in_pad, int32_t* hidden, int64_t* num_params) {
    if (!n) return LUDAX_ERR_ARG;
    if (in_pad) *in_pad = n->kpad;
    if (hidden) *hidden = kH;
    if (num_params) *num_params = n->nparams;
    return LUDAX_OK;
}

int ludax_net_set_params(ludax_net* n, const float* params_dev) {
    if (!n || !params_dev) return LUDAX_ERR_ARG;
    if (cudaMemcpyAsync(n->p, params_dev, sizeof(float) * n->nparams, cudaMemcpyDeviceToDevice, n->stream) != cudaSuccess ||
        cudaMemsetAsync(n->m, 0, sizeof(float) * n->nparams, n->stream) != cudaSuccess ||
        cudaMemsetAsync(n->v, 0, sizeof(float) * n->nparams, n->stream) != cudaSuccess)
        return LUDAX_ERR_CUDA;
    n->t = 0;
    return refresh_bf16(n);
}

int ludax_net_set_tensor_path(ludax_net* n, int32_t use_tcgen05) {
    if (!n || use_tcgen05 < 0 || use_tcgen05 > 2) return LUDAX_ERR_ARG;
    n->use_tcgen05 = use_tcgen05;
    return LUDAX_OK;
}

int ludax_net_get_params(ludax_net* n, float* params_dev) {
    if (!n || !params_dev) return LUDAX_ERR_ARG;
    return cudaMemcpyAsync(params_dev, n->p, sizeof(float) * n->nparams, cudaMemcpyDeviceToDevice, n->stream) == cudaSuccess
               ? LUDAX_OK
               : LUDAX_ERR_CUDA;
}

int ludax_net_get_state(ludax_net* n, float* params_dev, float* m_dev, float* v_dev, int64_t* steps) {
    if (!n) return LUDAX_ERR_ARG;
    const size_t bytes = sizeof(float) * (size_t)n->nparams;
    const float* src[3] = {n->p, n->m, n->v};
    float* dst[3] = {params_dev, m_dev, v_dev};
    for (int i = 0; i < 3; ++i)
        if (dst[i] && cudaMemcpyAsync(dst[i], src[i], bytes, cudaMemcpyDeviceToDevice, n->stream) != cudaSuccess)
            return LUDAX_ERR_CUDA;
    if (steps) *steps = n->t;
    return LUDAX_OK;
}

int ludax_net_set_state(ludax_net* n, const float* params_dev, const float* m_dev, const float* v_dev, int64_t steps) {
    if (!n || !params_dev || !m_dev || !v_dev || steps < 0 || steps > 0x7FFFFFFF) return LUDAX_ERR_ARG;
    const size_t bytes = sizeof(float) * (size_t)n->nparams;
    if (cudaMemcpyAsync(n->p, params_dev, bytes, cudaMemcpyDeviceToDevice, n->stream) != cudaSuccess ||
        cudaMemcpyAsync(n->m, m_dev, bytes, cudaMemcpyDeviceToDevice, n->stream) != cudaSuccess ||
        cudaMemcpyAsync(n->v, v_dev, bytes, cudaMemcpyDeviceToDevice, n->stream) != cudaSuccess)
        return LUDAX_ERR_CUDA;
    n->t = (int)steps;
    return refresh_bf16(n);  // the BF16 copies Adam leaves are the rounded parameters
}

int ludax_net_forward(ludax_net* n, const uint16_t* x_dev, int64_t B, float* p_dev) {
    ludax::ApiRange api_range("ludax_net_forward");
    int st = net_check(n, B);
    if (st) return st;
    if (!x_dev || !p_dev) return LUDAX_ERR_ARG;
    if ((uintptr_t)x_dev % 16) return LUDAX_ERR_ALIGN;
    return net_forward(n, reinterpret_cast<const __nv_bfloat16*>(x_dev), B, p_dev, nullptr);
}

int ludax_net_grad(ludax_net* n, const uint16_t* x_dev, const float* y_dev, int64_t B, float* grad_dev, float* loss_dev) {
    ludax::ApiRange api_range("ludax_net_grad");
    int st = net_check(n, B);
    if (st) return st;
    if (!x_dev || !y_dev) return LUDAX_ERR_ARG;
    if ((uintptr_t)x_dev % 16) return LUDAX_ERR_ALIGN;
    const __nv_bfloat16* X = reinterpret_cast<const __nv_bfloat16*>(x_dev);
    if ((st = net_forward(n, X, B, n->pout, y_dev))) return st;
    if ((st = net_backward(n, X, B, y_dev, loss_dev, nullptr))) return st;
    if (grad_dev && cudaMemcpyAsync(grad_dev, n->g, sizeof(float) * n->nparams, cudaMemcpyDeviceToDevice, n->stream) != cudaSuccess)
        return LUDAX_ERR_CUDA;
    return LUDAX_OK;
}

int ludax_net_train_step(ludax_net* n, const uint16_t* x_dev, const float* y_dev, int64_t B, float lr, float* loss_dev) {
    ludax::ApiRange api_range("ludax_net_train_step");
    int st = net_check(n, B);
    if (st) return st;
    if (!x_dev || !y_dev) return LUDAX_ERR_ARG;
    if ((uintptr_t)x_dev % 16) return LUDAX_ERR_ALIGN;
    const __nv_bfloat16* X = reinterpret_cast<const __nv_bfloat16*>(x_dev);
    const int t = n->t + 1;
    const AdamStep adam{lr, 1.f - powf(0.9f, (float)t), 1.f - powf(0.999f, (float)t)};
    if ((st = net_forward(n, X, B, n->pout, y_dev))) return st;
    if ((st = net_backward(n, X, B, y_dev, loss_dev, &adam))) return st;
    n->t = t;
    return LUDAX_OK;
}

int ludax_pack_inputs(ludax_env* env, uint16_t* x_dev, int32_t ld) {
    ludax::ApiRange api_range("ludax_pack_inputs");
    if (!env || !x_dev || ld < 2 * env->cells + 1 || ld % 8) return LUDAX_ERR_ARG;
    if ((uintptr_t)x_dev % 16) return LUDAX_ERR_ALIGN;
    return dispatch_game(env->game, env->rows, env->cols, [&](auto tag) {
        using G = typename decltype(tag)::type;
        if constexpr (IsMove<G>::value) {
            return LUDAX_ERR_GAME;  // the value net encodes placement boards (two stone planes)
        } else {
        pack_inputs_kernel<G><<<blocks_for(env->n, 128), 128, 0, env->stream>>>(
            EnvDev{env->d_planes, env->d_meta, env->n, env->env_offset, env->d_counters, env->desc, env->cells},
            reinterpret_cast<__nv_bfloat16*>(x_dev), ld);
        return cudaGetLastError() == cudaSuccess ? LUDAX_OK : LUDAX_ERR_CUDA;
        }
    });
}

int ludax_truncated_value(ludax_env* env, ludax_net* n, uint64_t seed, int32_t K, int32_t plies, float* value_dev) {
    ludax::ApiRange api_range("ludax_truncated_value");
    if (!env || !n || !value_dev || K < 1 || plies < 0) return LUDAX_ERR_ARG;
    if (n->cells != env->cells) return LUDAX_ERR_SIZE;
    if (n->stream != env->stream) return LUDAX_ERR_ARG;
    long long chunk = (n->max_batch / K);
    if (chunk < 1) return LUDAX_ERR_SIZE;
    return dispatch_game(env->game, env->rows, env->cols, [&](auto tag) -> int {
        using G = typename decltype(tag)::type;
        if constexpr (IsMove<G>::value) {
            return LUDAX_ERR_GAME;  // the value net encodes placement boards (two stone planes)
        } else {
        EnvDev d{env->d_planes, env->d_meta, env->n, env->env_offset, env->d_counters, env->desc, env->cells};
        for (long long e0 = 0; e0 < env->n; e0 += chunk) {
            long long nc = std::min(chunk, env->n - e0);
            long long rows = nc * K, rows_pad = ((rows + BM - 1) / BM) * BM;
            // the first layer reads only the 64-column blocks that hold the
            // 2 * cells + 1 inputs; the leaf rows are written that far, and the
            // padding rows up to a multiple of 128 as zeros
            const int kuse = ((n->kin + 63) / 64) * 64;
            if (launch_dependent(leaf_kernel<G>, blocks_for(rows_pad, LEAF_THREADS), LEAF_THREADS, 0, env->stream, d,
                                 e0, nc, K, seed, plies, n->Xleaf, (int)n->kpad, kuse, n->score, n->done,
                                 rows_pad) != cudaSuccess)
                return LUDAX_ERR_CUDA;
            // with one or two continuations per position the mean takes each p from its head partials
            // (one launch instead of two); with more, a thread per continuation forms p first
            if (K <= 2 && infer_tc(n, rows_pad, kuse)) {
                const float* zpart;
                int parts;
                int st = infer_head(n, n->Xleaf, rows_pad, kuse, &zpart, &parts);
                if (st) return st;
                if (launch_dependent(combine_z_kernel, blocks_for(nc, 256), 256, 0, env->stream, e0, nc, K,
                                     (const float*)n->score, (const uint8_t*)n->done, zpart, parts,
                                     (const float*)(n->p + n->ob3), value_dev) != cudaSuccess)
                    return LUDAX_ERR_CUDA;
                continue;
            }
            int st = net_forward(n, n->Xleaf, rows_pad, n->pout, nullptr, kuse);
            if (st) return st;
            combine_kernel<<<blocks_for(nc, 256), 256, 0, env->stream>>>(e0, nc, K, n->score, n->done, n->pout, value_dev);
        }
        return cudaGetLastError() == cudaSuccess ? LUDAX_OK : LUDAX_ERR_CUDA;
        }
    });
}

}  // extern "C"
