// mlp.cu -- a small fitness-surrogate MLP trained and run on the 5th-generation
// tensor cores (tcgen05) with BF16 operands and FP32 accumulation.
//
// The surrogate predicts a robot's 1 s centroid displacement from its voxel
// occupancy and per-voxel actuation phases; it pre-screens mutants in a
// morphology search whose survivors the simulator then scores (the paper's
// Sec. III-F topology and actuation optimisation, with a learned filter).
// Network: in -> hidden -> hidden -> hidden -> 1, GELU after each hidden layer.
//
// GEMM kernel (k_gemm_tn): C[M, N] = A[M, K] * B[N, K]^T with A and B row-major
// BF16 (K contiguous).  One CTA per 128 x BN output tile (BN = 64, 128 or
// 256), optionally one K slice of it (split K), 256 threads:
//   warp 0 lane 0  - TMA producer: 2-D tiled loads (128-byte swizzle) of the
//                    A and B K-blocks (64 wide) into a 4-stage ring;
//   warp 1 lane 0  - MMA issuer: tcgen05.mma.kind::f16 (M = 128, N = BN,
//                    K = 16) into an FP32 accumulator in TMEM, releasing each
//                    stage with tcgen05.commit;
//   all 8 warps    - epilogue: tcgen05.ld of the accumulator (warp w reads
//                    TMEM lanes 32 (w mod 4) .. + 31 = output rows, half
//                    w / 4 of the columns), each 32 x 32 block staged in the
//                    idle stage buffers so that global traffic runs along rows:
//                    FP32 output, fused bias + GELU, or the GELU-derivative
//                    product of back-propagation, with optional transposed
//                    BF16 copies and bias-gradient column partials.
// Every mbarrier wait is bounded (spin_limit polls); on expiry the kernel sets
// *err, waits (bounded) for its own copies and products in flight, skips the
// epilogue, frees its TMEM and returns.
//
// Training step: one CUDA graph per batch size (forward, loss, backward with
// the weight-gradient products on a second stream, Adam), replayed by
// titan_mlp_train_step; the learning rate and the Adam step counter live in
// device memory so the replay needs no host values.
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <random>
#include <string>
#include <vector>

#include "ptx.cuh"
#include "titan.h"

namespace titan {
void set_thread_error(const std::string &msg);   // runtime.cu
}

namespace {

// BM x BN output tile per CTA; BN = 64, 128 or 256 (wide tiles for large
// products: each A tile then feeds twice the columns, halving the A traffic
// from L2 per FLOP).
constexpr int BM = 128, BN = 128, BK = 64, STAGES = 4;
// 8 warps: warps 0 and 1 issue the loads and the products; after the
// mainloop all 8 run the epilogue, warp w on TMEM lanes 32 (w mod 4) ..
// + 31 (the lanes its quarter may read) and on half w / 4 of the columns
constexpr int kGemmThreads = 256;
constexpr uint32_t kStageA = BM * BK * 2;
template <int BN_> constexpr uint32_t stage_b() { return (uint32_t)BN_ * BK * 2; }
template <int BN_> constexpr size_t gemm_smem() { return (size_t)STAGES * (kStageA + stage_b<BN_>()) + 1024; }

enum Epi { EPI_F32 = 0, EPI_BIAS_GELU = 1, EPI_GELU_GRAD = 2 };

struct EpiArgs {
    int mode;
    int ldc;                      // row stride of the outputs (elements)
    const float *bias;            // [N]            (BIAS_GELU)
    float *out_f32;               // [M, ldc]       (F32: C; BIAS_GELU: pre-activation Z)
    __nv_bfloat16 *out_bf16;      // [M, ldc]       (BIAS_GELU: GELU(Z); GELU_GRAD: dZ)
    const float *z;               // [M, ldc]       (GELU_GRAD: the forward pre-activation)
    __nv_bfloat16 *out_t = nullptr;   // [N, ldt] the transpose of out_bf16, if given (BIAS_GELU, GELU_GRAD)
    int ldt = 0;
    float *colsum = nullptr;          // [M / 32, ldc] GELU_GRAD: per 32 rows, the column sums of out_bf16
};

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// Instruction descriptor of tcgen05.mma.kind::f16: FP32 accumulator, BF16 A
// and B, both K-major, N = BN_, M = BM.
template <int BN_>
constexpr uint32_t idesc() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN_ >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

template <int BN_>
__global__ void __launch_bounds__(kGemmThreads, 1)
k_gemm_tn(const __grid_constant__ CUtensorMap tma_a, const __grid_constant__ CUtensorMap tma_b, int K, EpiArgs ep,
          uint32_t spin_limit, int *__restrict__ err) {
    extern __shared__ uint8_t gsm_raw[];
    __shared__ uint64_t full[STAGES], empty[STAGES], accf;
    __shared__ uint32_t tmem_base;
    __shared__ int failed;
    __shared__ int n_issued;                          // k blocks whose TMA loads were issued
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // 1024-byte aligned tiles (the 128-byte swizzle pattern repeats every 1024 bytes)
    const uint32_t raw = titan::ptx::smem_u32(gsm_raw);
    uint8_t *gsm = gsm_raw + (((raw + 1023u) & ~1023u) - raw);
    constexpr uint32_t kStageB = stage_b<BN_>();
    constexpr uint32_t kTmemCols = (uint32_t)BN_;      // one FP32 column per output column
    auto tileA = [&](int s) { return gsm + (size_t)s * (kStageA + kStageB); };
    auto tileB = [&](int s) { return gsm + (size_t)s * (kStageA + kStageB) + kStageA; };
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN_;
    // split K (gridDim.z slices): slice z multiplies columns [z K, (z + 1) K) of A
    // and B and writes its partial product to its own M x ldc block of out_f32
    const int num_kb = K / BK;
    const int k0 = (int)blockIdx.z * K;

    if (warp == 0) titan::ptx::tmem_alloc(&tmem_base, kTmemCols);
    if (tid == 32) {
        for (int s = 0; s < STAGES; ++s) {
            titan::ptx::mbar_init(&full[s], 1);
            titan::ptx::mbar_init(&empty[s], 1);
        }
        titan::ptx::mbar_init(&accf, 1);
        titan::ptx::fence_mbar_init();
        failed = 0;
        n_issued = 0;
    }
    titan::ptx::tc_fence_before();
    __syncthreads();
    titan::ptx::tc_fence_after();
    const uint32_t taddr = tmem_base;

    if (warp == 0 && lane == 0) {                      // TMA producer
        for (int kb = 0; kb < num_kb; ++kb) {
            const int s = kb % STAGES;
            const uint32_t use = kb / STAGES;
            if (kb >= STAGES && !titan::ptx::mbar_wait_bounded(&empty[s], (use & 1) ^ 1, spin_limit)) {
                atomicExch(&failed, 1);
                break;
            }
            titan::ptx::mbar_arrive_expect_tx(&full[s], kStageA + kStageB);
            titan::ptx::tma_load_2d(tileA(s), &tma_a, k0 + kb * BK, m0, &full[s]);
            titan::ptx::tma_load_2d(tileB(s), &tma_b, k0 + kb * BK, n0, &full[s]);
            n_issued = kb + 1;
        }
    } else if (warp == 1 && lane == 0) {               // MMA issuer
        bool ok = true;
        for (int kb = 0; kb < num_kb && ok; ++kb) {
            const int s = kb % STAGES;
            if (!titan::ptx::mbar_wait_bounded(&full[s], (kb / STAGES) & 1, spin_limit)) {
                atomicExch(&failed, 1);
                ok = false;
                break;
            }
            titan::ptx::tc_fence_after();
            const uint32_t a0 = titan::ptx::smem_u32(tileA(s)), b0 = titan::ptx::smem_u32(tileB(s));
#pragma unroll
            for (int k = 0; k < BK / 16; ++k)
                titan::ptx::tc_mma_bf16(taddr, titan::ptx::smem_desc_sw128(a0 + 32 * k),
                                        titan::ptx::smem_desc_sw128(b0 + 32 * k), idesc<BN_>(), (kb | k) != 0);
            titan::ptx::tc_commit(&empty[s]);
        }
        titan::ptx::tc_commit(&accf);                  // fires when every issued MMA is done
    }
    __syncwarp();
    // epilogue: every thread owns one output row (its TMEM lane)
    const bool acc_ok = titan::ptx::mbar_wait_bounded(&accf, 0, spin_limit);
    titan::ptx::tc_fence_after();
    __syncthreads();
    if (!acc_ok || failed) {
        // a bounded wait expired: record it, then wait (bounded again) for
        // this CTA's own copies and products still in flight - the last TMA
        // load issued on each stage and every committed MMA - before the
        // tensor memory is freed and the CTA exits
        if (tid == 0) {
            // a plain store: the flag may live in pinned host memory
            *reinterpret_cast<volatile int *>(err) = 1;
            __threadfence_system();
            for (int st = 0; st < STAGES; ++st) {
                int last = -1;
                for (int kb = st; kb < n_issued; kb += STAGES) last = kb;
                if (last >= 0) titan::ptx::mbar_wait_bounded(&full[st], (uint32_t)(last / STAGES) & 1u, spin_limit);
            }
            if (!acc_ok) titan::ptx::mbar_wait_bounded(&accf, 0, spin_limit);
        }
        __syncthreads();
    } else {
        // The accumulator comes out of TMEM one row per lane.  Each 32 x 32
        // block goes through this warp's scratch in the (now idle) stage
        // buffers so that global reads and writes run along rows (lane =
        // column, 128-byte lines), and the transposed copy, if any, along
        // its columns (lane = row).
        float *scr = reinterpret_cast<float *>(gsm) + warp * (32 * 33);
        const int quarter = (int)(warp & 3), half = (int)(warp >> 2);
        const int row0 = m0 + quarter * 32;
        const size_t zoff = (size_t)blockIdx.z * gridDim.y * BM * ep.ldc;   // split-K slice (EPI_F32)
        for (int c0 = half * (BN_ / 2); c0 < (half + 1) * (BN_ / 2); c0 += 32) {
            float v[32];
            titan::ptx::tmem_ld32(taddr + (((uint32_t)quarter * 32u) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int k = 0; k < 32; ++k) scr[lane * 33 + k] = v[k];
            __syncwarp();
            const int col = n0 + c0 + lane;
            if (ep.mode == EPI_F32) {
#pragma unroll 8
                for (int r = 0; r < 32; ++r) ep.out_f32[zoff + (size_t)(row0 + r) * ep.ldc + col] = scr[r * 33 + lane];
            } else {
                if (ep.mode == EPI_BIAS_GELU) {
                    const float b = ep.bias[col];
#pragma unroll 8
                    for (int r = 0; r < 32; ++r) {
                        const size_t o = (size_t)(row0 + r) * ep.ldc + col;
                        const float z = scr[r * 33 + lane] + b;
                        ep.out_f32[o] = z;
                        const __nv_bfloat16 hb = __float2bfloat16_rn(gelu(z));
                        ep.out_bf16[o] = hb;
                        scr[r * 33 + lane] = __bfloat162float(hb);     // exact: read back for the transpose
                    }
                } else {
                    // the block's 32 rows of Z requested together, then the products;
                    // the column sums of the BF16 results (rows in order) feed the bias gradient
                    float zr[32];
#pragma unroll
                    for (int r = 0; r < 32; ++r) zr[r] = ep.z[(size_t)(row0 + r) * ep.ldc + col];
                    float cs = 0.f;
#pragma unroll
                    for (int r = 0; r < 32; ++r) {
                        const size_t o = (size_t)(row0 + r) * ep.ldc + col;
                        const __nv_bfloat16 hb = __float2bfloat16_rn(scr[r * 33 + lane] * gelu_grad(zr[r]));
                        ep.out_bf16[o] = hb;
                        const float hf = __bfloat162float(hb);
                        cs += hf;
                        scr[r * 33 + lane] = hf;                        // exact: read back for the transpose
                    }
                    if (ep.colsum) ep.colsum[(size_t)(row0 >> 5) * ep.ldc + col] = cs;
                }
                if (ep.out_t) {
                    __syncwarp();
#pragma unroll 8
                    for (int k = 0; k < 32; ++k)
                        ep.out_t[(size_t)(n0 + c0 + k) * ep.ldt + row0 + lane] = __float2bfloat16_rn(scr[lane * 33 + k]);
                }
            }
            __syncwarp();
        }
    }
    titan::ptx::tc_fence_before();
    __syncthreads();
    if (warp == 0) titan::ptx::tmem_dealloc(taddr, kTmemCols);
}

// ------------------------------------------------------------------ CUDA-core kernels

// out[c][r] = in[r][c] for a rows x cols BF16 matrix (32 x 32 tiles through shared memory).
__global__ void k_transpose_bf16(const __nv_bfloat16 *__restrict__ in, __nv_bfloat16 *__restrict__ out, int rows,
                                 int cols) {
    __shared__ __nv_bfloat16 t[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int r = by + k, c = bx + threadIdx.x;
        if (r < rows && c < cols) t[k][threadIdx.x] = in[(size_t)r * cols + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int c = bx + k, r = by + threadIdx.x;
        if (r < rows && c < cols) out[(size_t)c * rows + r] = t[threadIdx.x][k];
    }
}

// out[c][r] = in[r][c] for a rows x cols BF16 matrix, both multiples of 64
// and 16-byte aligned: 64 x 64 tiles, 16-byte global loads and stores (256
// threads).  Tile rows are 37 words apart in shared memory, so the eight
// input rows a warp gathers for one output vector fall in different banks.
__global__ void __launch_bounds__(256) k_transpose64_bf16(const __nv_bfloat16 *__restrict__ in,
                                                          __nv_bfloat16 *__restrict__ out, int rows, int cols) {
    constexpr int kW = 37;                              // words per tile row (64 values + 5 words pad)
    __shared__ uint32_t t[64 * kW];
    const int c0 = blockIdx.x * 64, r0 = blockIdx.y * 64, tid = threadIdx.x;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int q = tid + 256 * h, r = q >> 3, seg = (q & 7) * 8;
        const uint4 v = *reinterpret_cast<const uint4 *>(in + (size_t)(r0 + r) * cols + c0 + seg);
        uint32_t *d = t + r * kW + seg / 2;
        d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
    }
    __syncthreads();
    const __nv_bfloat16 *tb = reinterpret_cast<const __nv_bfloat16 *>(t);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int q = tid + 256 * h, c = q >> 3, seg = (q & 7) * 8;   // output row c, input rows seg..seg+7
        __align__(16) __nv_bfloat16 o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) o[k] = tb[(seg + k) * (2 * kW) + c];
        *reinterpret_cast<uint4 *>(out + (size_t)(c0 + c) * rows + r0 + seg) = *reinterpret_cast<const uint4 *>(o);
    }
}

__global__ void k_f32_to_bf16(const float *__restrict__ in, __nv_bfloat16 *__restrict__ out, size_t n) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float2bfloat16_rn(in[i]);
}

// y[b] = H[b, :] . w + bias (one warp per row).
__global__ void k_out_layer(const __nv_bfloat16 *__restrict__ H, const float *__restrict__ w, const float *__restrict__ b,
                            float *__restrict__ y, int rows, int cols) {
    const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (row >= rows) return;
    float s = 0.f;
    for (int c = lane; c < cols; c += 32) s += __bfloat162float(H[(size_t)row * cols + c]) * w[c];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[row] = s + b[0];
}

constexpr int kLossThreads = 1024;

// dy = 2 (y - t) / B and the mean-squared error (one block, fixed order).
// The output bias's gradient db = sum_b dy[b] is reduced alongside, in the
// same fixed order.
// tick (training steps only): the device Adam step counter, advanced here.
__global__ void k_loss(const float *__restrict__ y, const float *__restrict__ t, float *__restrict__ dy,
                       float *__restrict__ loss, int B, float *__restrict__ db, unsigned long long *__restrict__ tick) {
    __shared__ float part[kLossThreads], pdb[kLossThreads];
    float s = 0.f, sd = 0.f;
#pragma unroll 8
    for (int i = threadIdx.x; i < B; i += kLossThreads) {
        const float d = y[i] - t[i];
        const float g = 2.f * d / (float)B;
        dy[i] = g;
        s += d * d;
        sd += g;
    }
    part[threadIdx.x] = s;
    pdb[threadIdx.x] = sd;
    __syncthreads();
    for (int o = kLossThreads / 2; o; o >>= 1) {
        if (threadIdx.x < o) {
            part[threadIdx.x] += part[threadIdx.x + o];
            pdb[threadIdx.x] += pdb[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (loss) *loss = part[0] / (float)B;
        if (db) *db = pdb[0];
        if (tick) *tick += 1;
    }
}

// Column reductions over the batch run in two fixed-order stages so that the
// whole GPU takes part: stage one sums chunks of kRowChunk rows per column
// (grid: column blocks x row chunks), stage two adds the chunk sums in order.
constexpr int kRowChunk = 32;

// Output layer backward, stage one: per (chunk, column) the partial of
// dw[c] = sum_b dy[b] H[b, c]; elementwise dZ[b, c] = dy[b] w[c] GELU'(Z[b, c])
// in BF16; and per (chunk, column) the partial column sum of that BF16 dZ
// (the last hidden layer's bias gradient).
__global__ void k_out_backward(const __nv_bfloat16 *__restrict__ H, const float *__restrict__ Z, const float *__restrict__ dy,
                               const float *__restrict__ w, float *__restrict__ part, __nv_bfloat16 *__restrict__ dZ,
                               float *__restrict__ part_b, int B, int cols) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (c >= cols) return;
    const int b0 = k * kRowChunk;               // B is a multiple of 128: every chunk is whole
    const float wc = w[c];
    // the chunk's loads first (all in flight together), then the arithmetic
    float hv[kRowChunk], zv[kRowChunk];
#pragma unroll
    for (int r = 0; r < kRowChunk; ++r) {
        const size_t o = (size_t)(b0 + r) * cols + c;
        hv[r] = __bfloat162float(H[o]);
        zv[r] = Z[o];
    }
    float s = 0.f, sb = 0.f;
#pragma unroll
    for (int r = 0; r < kRowChunk; ++r) {
        const float d = dy[b0 + r];
        s += d * hv[r];
        const __nv_bfloat16 g = __float2bfloat16_rn(d * wc * gelu_grad(zv[r]));
        dZ[(size_t)(b0 + r) * cols + c] = g;
        sb += __bfloat162float(g);
    }
    part[(size_t)k * cols + c] = s;
    part_b[(size_t)k * cols + c] = sb;
}

// Stage two: out[c] = the sum over chunks of part[k][c], in a fixed order:
// thread (c, j) of a 32 x 32 block adds chunks j, j + 32, ... in turn, then
// the 32 partial sums of a column are added pairwise in a fixed tree.
__global__ void __launch_bounds__(1024) k_col_sum_final(const float *__restrict__ part, int chunks, int cols,
                                                        float *__restrict__ out) {
    __shared__ float t[32][33];
    const int c = blockIdx.x * 32 + threadIdx.x, j = threadIdx.y;
    float s = 0.f;
    if (c < cols) {
#pragma unroll 4
        for (int k = j; k < chunks; k += 32) s += part[(size_t)k * cols + c];
    }
    t[j][threadIdx.x] = s;
    __syncthreads();
    for (int o = 16; o; o >>= 1) {
        if (j < o) t[j][threadIdx.x] += t[j + o][threadIdx.x];
        __syncthreads();
    }
    if (j == 0 && c < cols) out[c] = t[0][threadIdx.x];
}

// out[i] = sum over z of part[z][i], z in order (a split-K product's
// slices); four entries per thread (n a multiple of 4, arrays 16-byte aligned).
__global__ void k_sum_splits(float *__restrict__ out, const float *__restrict__ part, int splits, size_t n) {
    const size_t i = 4 * (blockIdx.x * (size_t)blockDim.x + threadIdx.x);
    if (i >= n) return;
    float4 s = *reinterpret_cast<const float4 *>(part + i);
    for (int z = 1; z < splits; ++z) {
        const float4 q = *reinterpret_cast<const float4 *>(part + (size_t)z * n + i);
        s.x += q.x; s.y += q.y; s.z += q.z; s.w += q.w;
    }
    *reinterpret_cast<float4 *>(out + i) = s;
}

// Adam (beta1, beta2, eps; bias corrections c1 = 1 - b1^t, c2 = 1 - b2^t)
// on parameter i: updates m, v and p, returns the new p.
struct AdamArgs {
    float *p;
    const float *g;
    float *m, *v;
    const float *lr;                      // device: a captured step reads the current rate
    const unsigned long long *t;          // device step counter (advanced by k_loss of the same step)
    float b1, b2, eps;
};

__device__ __forceinline__ float adam_one(const AdamArgs &a, size_t i, float c1, float c2, float lr) {
    const float gi = a.g[i];
    const float mi = a.b1 * a.m[i] + (1.f - a.b1) * gi;
    const float vi = a.b2 * a.v[i] + (1.f - a.b2) * gi * gi;
    a.m[i] = mi;
    a.v[i] = vi;
    const float pi = a.p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + a.eps);
    a.p[i] = pi;
    return pi;
}

// The three weight matrices W_l^T ([hid][in_l] at off_w[l], blockIdx.z = l),
// 32 x 32 tiles: Adam on every entry, then the BF16 copies the next step's
// products read - W^T itself (wt, same layout) and W (w, [in_l][hid], the
// tile transposed through shared memory) - written coalesced.  Blocks of
// blockIdx.z = 3 take the vectors (b1, b2, and b3, w4, b4: three ranges from
// voff, of rows, rows and 2 rows + 1 entries), 256 entries per block.
struct AdamW {
    uint32_t off[3], cols[3];
    __nv_bfloat16 *wt[3], *w[3];
    uint32_t rows;
    uint32_t voff[3];
};

__global__ void k_adam_w(AdamArgs a, AdamW W) {
    __shared__ __nv_bfloat16 tile[32][34];
    // the layer's fields picked without indexing the parameter block at run time
    const uint32_t l = blockIdx.z, rows = W.rows;
    if (l == 3) {
        const uint32_t v = (blockIdx.y * gridDim.x + blockIdx.x) * 256 + threadIdx.y * 32 + threadIdx.x;
        if (v >= 4 * rows + 1) return;
        const float tf = (float)*a.t;
        const float c1 = 1.f - powf(a.b1, tf), c2 = 1.f - powf(a.b2, tf);
        const uint32_t i = v < rows ? W.voff[0] + v : (v < 2 * rows ? W.voff[1] + (v - rows) : W.voff[2] + (v - 2 * rows));
        adam_one(a, i, c1, c2, *a.lr);
        return;
    }
    const uint32_t cols = l == 0 ? W.cols[0] : (l == 1 ? W.cols[1] : W.cols[2]);
    const uint32_t off = l == 0 ? W.off[0] : (l == 1 ? W.off[1] : W.off[2]);
    __nv_bfloat16 *const wt = l == 0 ? W.wt[0] : (l == 1 ? W.wt[1] : W.wt[2]);
    __nv_bfloat16 *const wn = l == 0 ? W.w[0] : (l == 1 ? W.w[1] : W.w[2]);
    const uint32_t bx = blockIdx.x * 32, by = blockIdx.y * 32;
    if (bx >= cols || by >= rows) return;       // layers narrower than the grid
    const float tf = (float)*a.t;
    const float c1 = 1.f - powf(a.b1, tf), c2 = 1.f - powf(a.b2, tf), lr = *a.lr;
    for (uint32_t k = threadIdx.y; k < 32; k += 8) {
        const uint32_t r = by + k, c = bx + threadIdx.x;
        const size_t o = (size_t)r * cols + c;
        const __nv_bfloat16 h = __float2bfloat16_rn(adam_one(a, off + o, c1, c2, lr));
        wt[o] = h;
        tile[k][threadIdx.x] = h;
    }
    __syncthreads();
    for (uint32_t k = threadIdx.y; k < 32; k += 8) {
        const uint32_t c = bx + k, r = by + threadIdx.x;
        wn[(size_t)c * rows + r] = tile[threadIdx.x][k];
    }
}

// ------------------------------------------------------------------ host helpers

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// Tensor map of a row-major [rows, cols] BF16 matrix read in 64 x 128 boxes.
bool make_map(CUtensorMap *map, const void *base, uint64_t rows, uint64_t cols, uint32_t box_rows = 128) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * 2};
    const cuuint32_t box[2] = {BK, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// C[M, N] = A[M, K] B[N, K]^T with the given epilogue.  M, N multiples of 128,
// K a multiple of 64; A, B 16-byte aligned with row strides of K elements.
template <int BN_>
cudaError_t gemm_tn_launch(const CUtensorMap &ma, const CUtensorMap &mb, int M, int N, int K, const EpiArgs &ep,
                           cudaStream_t st, uint32_t spin_limit, int *err, int splits = 1) {
    static std::atomic<uint64_t> attr_set{0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (!(attr_set.load() & (1ull << (dev & 63)))) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_tn<BN_>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)gemm_smem<BN_>());
        if (e != cudaSuccess) return e;
        attr_set.fetch_or(1ull << (dev & 63));
    }
    dim3 grid(N / BN_, M / BM, splits);
    k_gemm_tn<BN_><<<grid, kGemmThreads, gemm_smem<BN_>(), st>>>(ma, mb, K / splits, ep, spin_limit, err);
    return cudaGetLastError();
}

// splits > 1 (EPI_F32 only): K is cut into `splits` equal slices, each a
// multiple of BK, whose partial products land in consecutive M x ldc blocks of
// ep.out_f32 (the caller sums them, k_sum_splits).
cudaError_t gemm_tn(const void *A, const void *B, int M, int N, int K, const EpiArgs &ep, cudaStream_t st,
                    uint32_t spin_limit, int *err, int splits = 1) {
    if (M % BM || N % BN || K % BK || M <= 0 || N <= 0 || K <= 0) return cudaErrorInvalidValue;
    if (splits < 1 || (splits > 1 && (ep.mode != EPI_F32 || (K / splits) % BK || K % splits)))
        return cudaErrorInvalidValue;
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15) return cudaErrorInvalidValue;
    // 256-wide tiles once there are at least two waves of them on 152 SMs;
    // 64-wide tiles when 128-wide ones (split-K slices included) would not
    // fill one wave: twice the CTAs, two resident per SM (97 KB of shared
    // memory each), so one CTA's epilogue overlaps another's products
    const int64_t tiles128 = (int64_t)(N / 128) * (M / BM) * splits;
    const bool wide = splits == 1 && N % 256 == 0 && (int64_t)(N / 256) * (M / BM) >= 2 * 152;
    const bool narrow = !wide && tiles128 <= 152;
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, M, K) || !make_map(&mb, B, N, K, wide ? 256 : (narrow ? 64 : 128)))
        return cudaErrorInvalidValue;
    if (wide) return gemm_tn_launch<256>(ma, mb, M, N, K, ep, st, spin_limit, err);
    if (narrow) return gemm_tn_launch<64>(ma, mb, M, N, K, ep, st, spin_limit, err, splits);
    return gemm_tn_launch<128>(ma, mb, M, N, K, ep, st, spin_limit, err, splits);
}

inline unsigned nblk(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ------------------------------------------------------------------ the MLP

struct titan_mlp {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    uint32_t in = 0, hid = 0;
    uint32_t spin_limit = 1u << 22;
    size_t n_params = 0;
    // parameters: [W1t (hid x in), b1, W2t (hid x hid), b2, W3t, b3, w4 (hid), b4 (1)]
    size_t off_w[3] = {0, 0, 0}, off_b[3] = {0, 0, 0}, off_w4 = 0, off_b4 = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *wt[3] = {nullptr, nullptr, nullptr};   // BF16 W^T (out x in): forward B operand
    __nv_bfloat16 *w[3] = {nullptr, nullptr, nullptr};    // BF16 W (in x out): backward B operand
    uint32_t cap = 0;                                      // batch capacity of the activations
    float *Z[3] = {nullptr, nullptr, nullptr};
    __nv_bfloat16 *H[3] = {nullptr, nullptr, nullptr};
    __nv_bfloat16 *dZ[3] = {nullptr, nullptr, nullptr};
    // transposes for the weight gradients: x^T, H_0^T and H_1^T (written by
    // the forward products' epilogues), dZ_l^T (one buffer, layer by layer)
    __nv_bfloat16 *xT = nullptr, *HT[2] = {nullptr, nullptr}, *bT = nullptr, *bT2 = nullptr;
    // the weight-gradient products run on a second stream beside the
    // input-gradient products (fork and join events per layer)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork[3] = {nullptr, nullptr, nullptr}, ev_join[3] = {nullptr, nullptr, nullptr};
    float *y = nullptr, *dy = nullptr;
    float *part = nullptr;                                 // column-reduction chunk sums [B / kRowChunk][hidden]
    float *partb = nullptr;                                // the same for the bias gradient of one layer
    float *wsk = nullptr;                                  // split-K partial weight gradients [splits][hid][in]
    size_t wsk_cap = 0;                                    // floats
    int *err = nullptr;
    // the training step replayed as one CUDA graph per batch size: it reads its
    // batch from gx / gt (the caller's arrays are copied there first) and the
    // learning rate and step count from device memory
    cudaStream_t capture = nullptr;
    std::map<uint32_t, cudaGraphExec_t> train_graph;
    bool graphs_ok = true;
    __nv_bfloat16 *gx = nullptr;
    float *gt = nullptr, *gloss = nullptr, *d_lr = nullptr;
    unsigned long long *d_step = nullptr;
    uint32_t g_cap = 0;
    float lr_set = -1.f;
    std::vector<void *> allocs;
    std::string error;
};

namespace {

titan_status mfail(titan_mlp *m, titan_status st, const std::string &msg) {
    if (m) m->error = msg;
    else titan::set_thread_error(msg);
    return st;
}

#define MLP_CK(m, call)                                                                          \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return mfail((m), e_ == cudaErrorMemoryAllocation ? TITAN_E_OOM : TITAN_E_CUDA,       \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                    \
    } while (0)

template <typename T>
cudaError_t malloc_t(titan_mlp *m, T **p, size_t count) {
    void *raw = nullptr;
    cudaError_t e = cudaMalloc(&raw, std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) {
        m->allocs.push_back(raw);
        *p = static_cast<T *>(raw);
    }
    return e;
}

uint32_t layer_in(const titan_mlp *m, int l) { return l == 0 ? m->in : m->hid; }

// K slices of a weight-gradient product (hid x in, summed over the batch B):
// its hid/128 x in/128 tiles alone fill a small part of the 152 SMs, so the
// batch is cut into up to 8 slices of at least 4 k-blocks while the tiles
// times the slices stay within one wave.
int wgrad_splits(uint32_t hid, uint32_t in, uint32_t B) {
    const uint32_t tiles = (hid / BM) * (in / 128);
    int s = 1;
    while (s < 8 && tiles * (uint32_t)(2 * s) <= 152 && B % (uint32_t)(2 * s * BK) == 0 && B / (2 * s) >= 4 * BK)
        s *= 2;
    return s;
}

// Refreshes both BF16 layouts of the hidden-layer weights from the FP32 master.
cudaError_t refresh_bf16(titan_mlp *m) {
    for (int l = 0; l < 3; ++l) {
        const size_t n = (size_t)m->hid * layer_in(m, l);
        k_f32_to_bf16<<<nblk(n, 256), 256, 0, m->stream>>>(m->p + m->off_w[l], m->wt[l], n);
        dim3 grid(nblk(layer_in(m, l), 32), nblk(m->hid, 32));
        k_transpose_bf16<<<grid, dim3(32, 8), 0, m->stream>>>(m->wt[l], m->w[l], (int)m->hid, (int)layer_in(m, l));
    }
    return cudaGetLastError();
}

// One Adam step on every parameter (at the step count k_loss advanced on the
// device) and the BF16 copies of the new weights, in one launch.
cudaError_t adam_step(titan_mlp *m) {
    AdamArgs a{m->p, m->g, m->m, m->v, m->d_lr, m->d_step, 0.9f, 0.999f, 1e-8f};
    AdamW W;
    // b1, b2 and (b3, w4, b4): the parameter layout keeps the last three contiguous
    W.voff[0] = (uint32_t)m->off_b[0];
    W.voff[1] = (uint32_t)m->off_b[1];
    W.voff[2] = (uint32_t)m->off_b[2];
    for (int l = 0; l < 3; ++l) {
        W.off[l] = (uint32_t)m->off_w[l];
        W.cols[l] = layer_in(m, l);
        W.wt[l] = m->wt[l];
        W.w[l] = m->w[l];
    }
    W.rows = m->hid;
    k_adam_w<<<dim3(std::max(m->in, m->hid) / 32, m->hid / 32, 4), dim3(32, 8), 0, m->stream>>>(a, W);
    return cudaGetLastError();
}

cudaError_t ensure_batch(titan_mlp *m, uint32_t B) {
    if (B <= m->cap) return cudaSuccess;
    cudaError_t e;
    for (int l = 0; l < 3; ++l) {
        if ((e = malloc_t(m, &m->Z[l], (size_t)B * m->hid)) != cudaSuccess) return e;
        if ((e = malloc_t(m, &m->H[l], (size_t)B * m->hid)) != cudaSuccess) return e;
        if ((e = malloc_t(m, &m->dZ[l], (size_t)B * m->hid)) != cudaSuccess) return e;
    }
    if ((e = malloc_t(m, &m->xT, (size_t)B * m->in)) != cudaSuccess) return e;
    if ((e = malloc_t(m, &m->HT[0], (size_t)B * m->hid)) != cudaSuccess) return e;
    if ((e = malloc_t(m, &m->HT[1], (size_t)B * m->hid)) != cudaSuccess) return e;
    if ((e = malloc_t(m, &m->bT, (size_t)B * m->hid)) != cudaSuccess) return e;
    if ((e = malloc_t(m, &m->bT2, (size_t)B * m->hid)) != cudaSuccess) return e;
    if ((e = malloc_t(m, &m->y, B)) != cudaSuccess) return e;
    if ((e = malloc_t(m, &m->dy, B)) != cudaSuccess) return e;
    if ((e = malloc_t(m, &m->part, (size_t)((B + kRowChunk - 1) / kRowChunk) * m->hid)) != cudaSuccess) return e;
    if ((e = malloc_t(m, &m->partb, (size_t)((B + kRowChunk - 1) / kRowChunk) * m->hid)) != cudaSuccess) return e;
    size_t ws = 0;
    for (int l = 0; l < 3; ++l)
        ws = std::max(ws, (size_t)wgrad_splits(m->hid, layer_in(m, l), B) * m->hid * layer_in(m, l));
    if (ws > m->wsk_cap) {
        if ((e = malloc_t(m, &m->wsk, ws)) != cudaSuccess) return e;
        m->wsk_cap = ws;
    }
    m->cap = B;
    return cudaSuccess;
}

// keep_t: also write H_0^T and H_1^T (the backward pass's weight gradients read them).
cudaError_t forward_pass(titan_mlp *m, const __nv_bfloat16 *x, uint32_t B, float *y, bool keep_t = false) {
    cudaError_t e;
    const __nv_bfloat16 *a = x;
    for (int l = 0; l < 3; ++l) {
        EpiArgs ep{EPI_BIAS_GELU, (int)m->hid, m->p + m->off_b[l], m->Z[l], m->H[l], nullptr};
        if (keep_t && l < 2) {
            ep.out_t = m->HT[l];
            ep.ldt = (int)B;
        }
        if ((e = gemm_tn(a, m->wt[l], (int)B, (int)m->hid, (int)layer_in(m, l), ep, m->stream, m->spin_limit, m->err)) != cudaSuccess)
            return e;
        a = m->H[l];
    }
    k_out_layer<<<nblk(B, 8), 256, 0, m->stream>>>(m->H[2], m->p + m->off_w4, m->p + m->off_b4, y, (int)B, (int)m->hid);
    return cudaGetLastError();
}

// train: a training step follows (k_loss advances the Adam step counter).
cudaError_t backward_pass(titan_mlp *m, const __nv_bfloat16 *x, const float *t, uint32_t B, float *loss,
                          bool train = false) {
    cudaError_t e = forward_pass(m, x, B, m->y, true);
    if (e != cudaSuccess) return e;
    k_loss<<<1, kLossThreads, 0, m->stream>>>(m->y, t, m->dy, loss, (int)B, m->g + m->off_b4,
                                              train ? m->d_step : nullptr);
    const int chunks = ((int)B + kRowChunk - 1) / kRowChunk;
    k_out_backward<<<dim3(nblk(m->hid, 128), chunks), 128, 0, m->stream>>>(m->H[2], m->Z[2], m->dy, m->p + m->off_w4,
                                                                          m->part, m->dZ[2], m->partb, (int)B,
                                                                          (int)m->hid);
    const dim3 cs_grid(nblk(m->hid, 32)), cs_block(32, 32);
    k_col_sum_final<<<cs_grid, cs_block, 0, m->stream>>>(m->part, chunks, (int)m->hid, m->g + m->off_w4);
    // dZ_l^T alternates between two buffers (layer 2 and 0: bT, layer 1: bT2),
    // so that layer l's weight-gradient product (second stream) can read its
    // own while the input-gradient product (this stream) writes the next
    __nv_bfloat16 *const bt[2] = {m->bT, m->bT2};
    k_transpose64_bf16<<<dim3(m->hid / 64, B / 64), 256, 0, m->stream>>>(m->dZ[2], bt[0], (int)B, (int)m->hid);
    for (int l = 2; l >= 0; --l) {
        // dW_l^T (hid x in_l) = dZ_l^T (hid x B) . A_{l-1}^T (in_l x B)^T, on the second stream
        const uint32_t in = layer_in(m, l);
        const __nv_bfloat16 *actT = l == 0 ? m->xT : m->HT[l - 1];
        if (l == 0)
            k_transpose64_bf16<<<dim3(in / 64, B / 64), 256, 0, m->stream>>>(x, m->xT, (int)B, (int)in);
        if ((e = cudaEventRecord(m->ev_fork[l], m->stream)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(m->side, m->ev_fork[l], 0)) != cudaSuccess) return e;
        const int splits = wgrad_splits(m->hid, in, B);
        EpiArgs ep{EPI_F32, (int)in, nullptr, splits > 1 ? m->wsk : m->g + m->off_w[l], nullptr, nullptr};
        if ((e = gemm_tn(bt[l & 1], actT, (int)m->hid, (int)in, (int)B, ep, m->side, m->spin_limit, m->err, splits)) !=
            cudaSuccess)
            return e;
        if (splits > 1) {
            const size_t n = (size_t)m->hid * in;
            k_sum_splits<<<nblk(n / 4, 256), 256, 0, m->side>>>(m->g + m->off_w[l], m->wsk, splits, n);
        }
        if ((e = cudaEventRecord(m->ev_join[l], m->side)) != cudaSuccess) return e;
        // db_l: the chunk sums of dZ_l's columns came with dZ_l (k_out_backward, or the
        // epilogue of the product that formed it); the next product overwrites them
        k_col_sum_final<<<cs_grid, cs_block, 0, m->stream>>>(m->partb, chunks, (int)m->hid, m->g + m->off_b[l]);
        if (l > 0) {
            // dZ_{l-1} = (dZ_l . W_l^T) * GELU'(Z_{l-1}):  A = dZ_l (B x hid), B operand = W_l (in x hid);
            // its transpose goes to the buffer layer l + 1's weight gradient read: wait for it
            if (l == 1 && (e = cudaStreamWaitEvent(m->stream, m->ev_join[2], 0)) != cudaSuccess) return e;
            EpiArgs ep2{EPI_GELU_GRAD, (int)m->hid, nullptr, nullptr, m->dZ[l - 1], m->Z[l - 1]};
            ep2.out_t = bt[(l - 1) & 1];
            ep2.ldt = (int)B;
            ep2.colsum = m->partb;
            if ((e = gemm_tn(m->dZ[l], m->w[l], (int)B, (int)in, (int)m->hid, ep2, m->stream, m->spin_limit, m->err)) != cudaSuccess)
                return e;
        }
    }
    // every weight gradient is in place before anything reads it (the side stream runs in order)
    if ((e = cudaStreamWaitEvent(m->stream, m->ev_join[0], 0)) != cudaSuccess) return e;
    return cudaGetLastError();
}

// One training step for a batch of B read from gx / gt, captured into a graph:
// the forward and backward products, the step counter, Adam, and the BF16
// copies of the new weights.
cudaError_t capture_train(titan_mlp *m, uint32_t B, cudaGraphExec_t *out) {
    cudaError_t e = cudaStreamBeginCapture(m->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaStream_t saved = m->stream;
    m->stream = m->capture;
    cudaError_t le = backward_pass(m, m->gx, m->gt, B, m->gloss, true);
    if (le == cudaSuccess) le = adam_step(m);
    m->stream = saved;
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(m->capture, &g);
    if (le != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return le != cudaSuccess ? le : e;
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return e;
}

void drop_train_graphs(titan_mlp *m) {
    for (auto &kv : m->train_graph) cudaGraphExecDestroy(kv.second);
    m->train_graph.clear();
}

titan_status check_err(titan_mlp *m) {
    int flag = 0;
    MLP_CK(m, cudaStreamSynchronize(m->stream));
    MLP_CK(m, cudaMemcpy(&flag, m->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        cudaMemset(m->err, 0, sizeof(int));
        return mfail(m, TITAN_E_TIMEOUT, "a bounded wait in the tensor-core GEMM expired");
    }
    return TITAN_OK;
}

}  // namespace

extern "C" {

// One bounded-wait flag per device ordinal for the standalone GEMM, in
// pinned host memory mapped into the device: a call reads it without
// waiting for its stream.
namespace {
std::mutex g_gemm_mu;
volatile int *g_gemm_flag[64] = {};
int *g_gemm_flag_dev[64] = {};

titan_status gemm_flag(int *dev_out, volatile int **host, int **dev_ptr, const char *who) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return mfail(nullptr, TITAN_E_CUDA, std::string(who) + ": no current device");
    std::lock_guard<std::mutex> lk(g_gemm_mu);
    if (!g_gemm_flag[dev]) {
        void *h = nullptr, *d = nullptr;
        if (cudaHostAlloc(&h, sizeof(int), cudaHostAllocMapped) != cudaSuccess)
            return mfail(nullptr, TITAN_E_OOM, std::string(who) + ": error flag");
        *static_cast<volatile int *>(h) = 0;
        if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
            cudaFreeHost(h);
            return mfail(nullptr, TITAN_E_CUDA, std::string(who) + ": error flag");
        }
        g_gemm_flag[dev] = static_cast<volatile int *>(h);
        g_gemm_flag_dev[dev] = static_cast<int *>(d);
    }
    *dev_out = dev;
    *host = g_gemm_flag[dev];
    *dev_ptr = g_gemm_flag_dev[dev];
    return TITAN_OK;
}
}  // namespace

titan_status titan_gemm_bf16_tn(uint32_t M, uint32_t N, uint32_t K, const uint16_t *A_dev, const uint16_t *B_dev,
                                float *C_dev, void *stream) {
    if (!A_dev || !B_dev || !C_dev) return mfail(nullptr, TITAN_E_INVALID, "titan_gemm_bf16_tn: null pointer");
    if (M % BM || N % BN || K % BK || !M || !N || !K)
        return mfail(nullptr, TITAN_E_INVALID, "titan_gemm_bf16_tn: M and N must be multiples of 128, K of 64");
    int dev = 0;
    volatile int *flag = nullptr;
    int *err = nullptr;
    titan_status fs = gemm_flag(&dev, &flag, &err, "titan_gemm_bf16_tn");
    if (fs != TITAN_OK) return fs;
    if (*flag) {                     // an earlier call's kernel gave up on a wait
        *flag = 0;
        return mfail(nullptr, TITAN_E_TIMEOUT, "titan_gemm_bf16_tn: a bounded wait expired in an earlier call");
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    EpiArgs ep{EPI_F32, (int)N, nullptr, C_dev, nullptr, nullptr};
    cudaError_t e = gemm_tn(A_dev, B_dev, (int)M, (int)N, (int)K, ep, st, 1u << 22, err);
    if (e != cudaSuccess) return mfail(nullptr, TITAN_E_CUDA, std::string("titan_gemm_bf16_tn: ") + cudaGetErrorString(e));
    return TITAN_OK;
}

titan_status titan_gemm_check(void) {
    int dev = 0;
    volatile int *flag = nullptr;
    int *err = nullptr;
    titan_status fs = gemm_flag(&dev, &flag, &err, "titan_gemm_check");
    if (fs != TITAN_OK) return fs;
    if (*flag) {
        *flag = 0;
        return mfail(nullptr, TITAN_E_TIMEOUT, "titan_gemm_bf16_tn: a bounded wait expired");
    }
    return TITAN_OK;
}

titan_status titan_mlp_create(uint32_t in, uint32_t hidden, uint64_t seed, int32_t device, void *stream,
                              titan_mlp **out) {
    if (!out || in % 128 || hidden % 128 || !in || !hidden)
        return mfail(nullptr, TITAN_E_INVALID, "titan_mlp_create: in and hidden must be positive multiples of 128");
    titan_mlp *m = new titan_mlp();
    m->device = device;
    m->in = in;
    m->hid = hidden;
    size_t o = 0;
    for (int l = 0; l < 3; ++l) {
        m->off_w[l] = o;
        o += (size_t)hidden * (l == 0 ? in : hidden);
        m->off_b[l] = o;
        o += hidden;
    }
    m->off_w4 = o;
    o += hidden;
    m->off_b4 = o;
    o += 1;
    m->n_params = o;
    auto bail = [&](titan_status st) {
        titan::set_thread_error(m->error);
        for (void *p : m->allocs) cudaFree(p);
        for (int l = 0; l < 3; ++l) {
            if (m->ev_fork[l]) cudaEventDestroy(m->ev_fork[l]);
            if (m->ev_join[l]) cudaEventDestroy(m->ev_join[l]);
        }
        if (m->side) cudaStreamDestroy(m->side);
        if (m->capture) cudaStreamDestroy(m->capture);
        if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
        delete m;
        return st;
    };
#define C_CK(call)                                                                               \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return bail(mfail(m, TITAN_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_))); \
    } while (0)
    C_CK(cudaSetDevice(device));
    if (!encode_fn()) return bail(mfail(m, TITAN_E_UNSUPPORTED, "cuTensorMapEncodeTiled is not available"));
    if (stream) m->stream = static_cast<cudaStream_t>(stream);
    else { C_CK(cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking)); m->own_stream = true; }
    C_CK(malloc_t(m, &m->p, o));
    C_CK(malloc_t(m, &m->g, o));
    C_CK(malloc_t(m, &m->m, o));
    C_CK(malloc_t(m, &m->v, o));
    C_CK(malloc_t(m, &m->err, 1));
    C_CK(malloc_t(m, &m->d_lr, 1));
    C_CK(malloc_t(m, &m->gloss, 1));
    C_CK(malloc_t(m, &m->d_step, 1));
    C_CK(cudaMemset(m->d_step, 0, sizeof(unsigned long long)));
    C_CK(cudaStreamCreateWithFlags(&m->capture, cudaStreamNonBlocking));
    C_CK(cudaStreamCreateWithFlags(&m->side, cudaStreamNonBlocking));
    for (int l = 0; l < 3; ++l) {
        C_CK(cudaEventCreateWithFlags(&m->ev_fork[l], cudaEventDisableTiming));
        C_CK(cudaEventCreateWithFlags(&m->ev_join[l], cudaEventDisableTiming));
    }
    for (int l = 0; l < 3; ++l) {
        C_CK(malloc_t(m, &m->wt[l], (size_t)hidden * layer_in(m, l)));
        C_CK(malloc_t(m, &m->w[l], (size_t)hidden * layer_in(m, l)));
    }
    // He-style initialisation (uniform, variance 2 / fan_in for GELU layers), zero biases
    std::vector<float> h(o, 0.f);
    std::mt19937_64 rng(seed);
    for (int l = 0; l < 3; ++l) {
        const float a = std::sqrt(6.0f / (float)layer_in(m, l));
        std::uniform_real_distribution<float> U(-a, a);
        for (size_t k = 0; k < (size_t)hidden * layer_in(m, l); ++k) h[m->off_w[l] + k] = U(rng);
    }
    {
        const float a = std::sqrt(3.0f / (float)hidden);
        std::uniform_real_distribution<float> U(-a, a);
        for (uint32_t k = 0; k < hidden; ++k) h[m->off_w4 + k] = U(rng);
    }
    C_CK(cudaMemcpy(m->p, h.data(), o * 4, cudaMemcpyHostToDevice));
    C_CK(cudaMemset(m->m, 0, o * 4));
    C_CK(cudaMemset(m->v, 0, o * 4));
    C_CK(cudaMemset(m->g, 0, o * 4));
    C_CK(cudaMemset(m->err, 0, sizeof(int)));
    C_CK(refresh_bf16(m));
    C_CK(cudaStreamSynchronize(m->stream));
#undef C_CK
    *out = m;
    return TITAN_OK;
}

uint64_t titan_mlp_param_count(const titan_mlp *m) { return m ? m->n_params : 0; }

titan_status titan_mlp_get_params(titan_mlp *m, float *host) {
    if (!m || !host) return TITAN_E_INVALID;
    MLP_CK(m, cudaStreamSynchronize(m->stream));
    MLP_CK(m, cudaMemcpy(host, m->p, m->n_params * 4, cudaMemcpyDeviceToHost));
    return TITAN_OK;
}

titan_status titan_mlp_set_params(titan_mlp *m, const float *host) {
    if (!m || !host) return TITAN_E_INVALID;
    MLP_CK(m, cudaStreamSynchronize(m->stream));
    MLP_CK(m, cudaMemcpy(m->p, host, m->n_params * 4, cudaMemcpyHostToDevice));
    MLP_CK(m, refresh_bf16(m));
    return check_err(m);
}

titan_status titan_mlp_forward(titan_mlp *m, const uint16_t *x_dev, uint32_t batch, float *y_dev) {
    if (!m || !x_dev || !y_dev || batch % 128 || !batch)
        return mfail(m, TITAN_E_INVALID, "titan_mlp_forward: batch must be a positive multiple of 128");
    MLP_CK(m, cudaSetDevice(m->device));
    MLP_CK(m, ensure_batch(m, batch));
    MLP_CK(m, forward_pass(m, reinterpret_cast<const __nv_bfloat16 *>(x_dev), batch, y_dev));
    return check_err(m);
}

titan_status titan_mlp_gradient(titan_mlp *m, const uint16_t *x_dev, const float *t_dev, uint32_t batch,
                                float *loss_dev, float *grad_dev) {
    if (!m || !x_dev || !t_dev || batch % 128 || !batch)
        return mfail(m, TITAN_E_INVALID, "titan_mlp_gradient: batch must be a positive multiple of 128");
    MLP_CK(m, cudaSetDevice(m->device));
    MLP_CK(m, ensure_batch(m, batch));
    MLP_CK(m, backward_pass(m, reinterpret_cast<const __nv_bfloat16 *>(x_dev), t_dev, batch, loss_dev));
    if (grad_dev) MLP_CK(m, cudaMemcpyAsync(grad_dev, m->g, m->n_params * 4, cudaMemcpyDeviceToDevice, m->stream));
    return check_err(m);
}

titan_status titan_mlp_train_step(titan_mlp *m, const uint16_t *x_dev, const float *t_dev, uint32_t batch, float lr,
                                  float *loss_dev) {
    if (!m || !x_dev || !t_dev || batch % 128 || !batch)
        return mfail(m, TITAN_E_INVALID, "titan_mlp_train_step: batch must be a positive multiple of 128");
    MLP_CK(m, cudaSetDevice(m->device));
    const uint32_t cap0 = m->cap;
    MLP_CK(m, ensure_batch(m, batch));
    if (m->cap != cap0) drop_train_graphs(m);           // the activations moved
    if (lr != m->lr_set) {                              // pageable source: staged before the call returns
        MLP_CK(m, cudaMemcpyAsync(m->d_lr, &lr, sizeof(float), cudaMemcpyHostToDevice, m->stream));
        m->lr_set = lr;
    }
    if (m->graphs_ok) {
        if (batch > m->g_cap) {
            drop_train_graphs(m);
            MLP_CK(m, malloc_t(m, &m->gx, (size_t)batch * m->in));
            MLP_CK(m, malloc_t(m, &m->gt, batch));
            m->g_cap = batch;
        }
        auto it = m->train_graph.find(batch);
        if (it == m->train_graph.end()) {
            cudaGraphExec_t ge = nullptr;
            if (capture_train(m, batch, &ge) == cudaSuccess) {
                it = m->train_graph.emplace(batch, ge).first;
            } else {                                    // capture refused: launch the kernels directly
                cudaGetLastError();
                m->graphs_ok = false;
            }
        }
        if (m->graphs_ok) {
            MLP_CK(m, cudaMemcpyAsync(m->gx, x_dev, (size_t)batch * m->in * 2, cudaMemcpyDeviceToDevice, m->stream));
            MLP_CK(m, cudaMemcpyAsync(m->gt, t_dev, (size_t)batch * 4, cudaMemcpyDeviceToDevice, m->stream));
            MLP_CK(m, cudaGraphLaunch(it->second, m->stream));
            if (loss_dev) MLP_CK(m, cudaMemcpyAsync(loss_dev, m->gloss, 4, cudaMemcpyDeviceToDevice, m->stream));
            return TITAN_OK;
        }
    }
    MLP_CK(m, backward_pass(m, reinterpret_cast<const __nv_bfloat16 *>(x_dev), t_dev, batch, loss_dev, true));
    MLP_CK(m, adam_step(m));
    return TITAN_OK;
}

titan_status titan_mlp_sync(titan_mlp *m) { return m ? check_err(m) : TITAN_E_INVALID; }

const char *titan_mlp_last_error(const titan_mlp *m) { return m ? m->error.c_str() : ""; }

titan_status titan_mlp_destroy(titan_mlp *m) {
    if (!m) return TITAN_OK;
    cudaStreamSynchronize(m->stream);
    if (m->side) cudaStreamSynchronize(m->side);
    drop_train_graphs(m);
    for (int l = 0; l < 3; ++l) {
        if (m->ev_fork[l]) cudaEventDestroy(m->ev_fork[l]);
        if (m->ev_join[l]) cudaEventDestroy(m->ev_join[l]);
    }
    if (m->side) cudaStreamDestroy(m->side);
    if (m->capture) cudaStreamDestroy(m->capture);
    for (void *p : m->allocs) cudaFree(p);
    if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
    delete m;
    return TITAN_OK;
}

}  // extern "C"
