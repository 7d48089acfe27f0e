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
// BF16 (K contiguous).  One CTA per 128 x 128 output tile, 128 threads:
//   warp 0 lane 0  - TMA producer: 2-D tiled loads (128-byte swizzle) of the
//                    A and B K-blocks (64 wide) into a 4-stage ring;
//   warp 1 lane 0  - MMA issuer: tcgen05.mma.kind::f16 (M = N = 128, K = 16)
//                    into an FP32 accumulator in TMEM, releasing each stage
//                    with tcgen05.commit;
//   all 4 warps    - epilogue: tcgen05.ld of the accumulator (warp w owns TMEM
//                    lanes 32w..32w+31 = output rows), fused bias + GELU, or
//                    the GELU-derivative product of back-propagation, stored
//                    to global memory.
// Every mbarrier wait is bounded (spin_limit polls); on expiry the kernel sets
// *err, skips the epilogue, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <atomic>
#include <cmath>
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

// BM x BN output tile per CTA; BN = 128 or 256 (wide tiles for large
// products: each A tile then feeds twice the columns, halving the A traffic
// from L2 per FLOP).
constexpr int BM = 128, BN = 128, BK = 64, STAGES = 4;
constexpr int kGemmThreads = 128;
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
    const int num_kb = K / BK;

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
            titan::ptx::tma_load_2d(tileA(s), &tma_a, kb * BK, m0, &full[s]);
            titan::ptx::tma_load_2d(tileB(s), &tma_b, kb * BK, n0, &full[s]);
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
            atomicExch(err, 1);
            for (int st = 0; st < STAGES; ++st) {
                int last = -1;
                for (int kb = st; kb < n_issued; kb += STAGES) last = kb;
                if (last >= 0) titan::ptx::mbar_wait_bounded(&full[st], (uint32_t)(last / STAGES) & 1u, spin_limit);
            }
            if (!acc_ok) titan::ptx::mbar_wait_bounded(&accf, 0, spin_limit);
        }
        __syncthreads();
    } else {
        const int row = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < BN_; c0 += 32) {
            float v[32];
            titan::ptx::tmem_ld32(taddr + ((warp * 32u) << 16) + (uint32_t)c0, v);
            const int col = n0 + c0;
            const size_t off = (size_t)row * ep.ldc + col;
            if (ep.mode == EPI_F32) {
#pragma unroll
                for (int k = 0; k < 32; k += 4)
                    *reinterpret_cast<float4 *>(ep.out_f32 + off + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
            } else if (ep.mode == EPI_BIAS_GELU) {
#pragma unroll
                for (int k = 0; k < 32; k += 2) {
                    const float z0 = v[k] + ep.bias[col + k], z1 = v[k + 1] + ep.bias[col + k + 1];
                    *reinterpret_cast<float2 *>(ep.out_f32 + off + k) = make_float2(z0, z1);
                    *reinterpret_cast<__nv_bfloat162 *>(ep.out_bf16 + off + k) = __floats2bfloat162_rn(gelu(z0), gelu(z1));
                }
            } else {
#pragma unroll
                for (int k = 0; k < 32; k += 2) {
                    const float2 z = *reinterpret_cast<const float2 *>(ep.z + off + k);
                    *reinterpret_cast<__nv_bfloat162 *>(ep.out_bf16 + off + k) =
                        __floats2bfloat162_rn(v[k] * gelu_grad(z.x), v[k + 1] * gelu_grad(z.y));
                }
            }
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

// dy = 2 (y - t) / B and the mean-squared error (one block, fixed order).
__global__ void k_loss(const float *__restrict__ y, const float *__restrict__ t, float *__restrict__ dy,
                       float *__restrict__ loss, int B) {
    __shared__ float part[256];
    float s = 0.f;
    for (int i = threadIdx.x; i < B; i += 256) {
        const float d = y[i] - t[i];
        dy[i] = 2.f * d / (float)B;
        s += d * d;
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss) *loss = part[0] / (float)B;
}

// Column reductions over the batch run in two fixed-order stages so that the
// whole GPU takes part: stage one sums chunks of kRowChunk rows per column
// (grid: column blocks x row chunks), stage two adds the chunk sums in order.
constexpr int kRowChunk = 64;

// Output layer backward, stage one: per (chunk, column) the partial of
// dw[c] = sum_b dy[b] H[b, c]; and, elementwise, dZ[b, c] = dy[b] w[c] GELU'(Z[b, c]) in BF16.
__global__ void k_out_backward(const __nv_bfloat16 *__restrict__ H, const float *__restrict__ Z, const float *__restrict__ dy,
                               const float *__restrict__ w, float *__restrict__ part, __nv_bfloat16 *__restrict__ dZ,
                               int B, int cols) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (c >= cols) return;
    const int b0 = k * kRowChunk, b1 = min(B, b0 + kRowChunk);
    const float wc = w[c];
    float s = 0.f;
    for (int b = b0; b < b1; ++b) {
        const size_t o = (size_t)b * cols + c;
        const float d = dy[b];
        s += d * __bfloat162float(H[o]);
        dZ[o] = __float2bfloat16_rn(d * wc * gelu_grad(Z[o]));
    }
    part[(size_t)k * cols + c] = s;
}

// Stage one of the bias gradients: per (chunk, column) the partial column sum of a BF16 [B, cols] matrix.
__global__ void k_col_sum_part(const __nv_bfloat16 *__restrict__ M, float *__restrict__ part, int B, int cols) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (c >= cols) return;
    const int b0 = k * kRowChunk, b1 = min(B, b0 + kRowChunk);
    float s = 0.f;
    for (int b = b0; b < b1; ++b) s += __bfloat162float(M[(size_t)b * cols + c]);
    part[(size_t)k * cols + c] = s;
}

// Stage two: out[c] = sum over chunks, in chunk order; thread `cols` also
// forms db = sum_b dy[b] when dy is given (the output bias).
__global__ void k_col_sum_final(const float *__restrict__ part, int chunks, int cols, float *__restrict__ out,
                                const float *__restrict__ dy, int B, float *__restrict__ db) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < cols) {
        float s = 0.f;
        for (int k = 0; k < chunks; ++k) s += part[(size_t)k * cols + c];
        out[c] = s;
    } else if (c == cols && dy) {
        float s = 0.f;
        for (int b = 0; b < B; ++b) s += dy[b];
        db[0] = s;
    }
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       size_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
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
                           cudaStream_t st, uint32_t spin_limit, int *err) {
    static std::atomic<uint64_t> attr_set{0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (!(attr_set.load() & (1ull << (dev & 63)))) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_tn<BN_>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)gemm_smem<BN_>());
        if (e != cudaSuccess) return e;
        attr_set.fetch_or(1ull << (dev & 63));
    }
    dim3 grid(N / BN_, M / BM);
    k_gemm_tn<BN_><<<grid, kGemmThreads, gemm_smem<BN_>(), st>>>(ma, mb, K, ep, spin_limit, err);
    return cudaGetLastError();
}

cudaError_t gemm_tn(const void *A, const void *B, int M, int N, int K, const EpiArgs &ep, cudaStream_t st,
                    uint32_t spin_limit, int *err) {
    if (M % BM || N % BN || K % BK || M <= 0 || N <= 0 || K <= 0) return cudaErrorInvalidValue;
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15) return cudaErrorInvalidValue;
    // 256-wide tiles once there are at least two waves of them on 152 SMs
    const bool wide = N % 256 == 0 && (int64_t)(N / 256) * (M / BM) >= 2 * 152;
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, M, K) || !make_map(&mb, B, N, K, wide ? 256 : 128)) return cudaErrorInvalidValue;
    return wide ? gemm_tn_launch<256>(ma, mb, M, N, K, ep, st, spin_limit, err)
                : gemm_tn_launch<128>(ma, mb, M, N, K, ep, st, spin_limit, err);
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
    __nv_bfloat16 *xT = nullptr, *aT = nullptr, *bT = nullptr;   // transposes for weight gradients
    float *y = nullptr, *dy = nullptr;
    float *part = nullptr;                                 // column-reduction chunk sums [B / kRowChunk][hidden]
    int *err = nullptr;
    uint64_t adam_t = 0;
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

cudaError_t ensure_batch(titan_mlp *m, uint32_t B) {
    if (B <= m->cap) return cudaSuccess;
    cudaError_t e;
    for (int l = 0; l < 3; ++l) {
        if ((e = malloc_t(m, &m->Z[l], (size_t)B * m->hid)) != cudaSuccess) return e;
        if ((e = malloc_t(m, &m->H[l], (size_t)B * m->hid)) != cudaSuccess) return e;
        if ((e = malloc_t(m, &m->dZ[l], (size_t)B * m->hid)) != cudaSuccess) return e;
    }
    if ((e = malloc_t(m, &m->xT, (size_t)B * m->in)) != cudaSuccess) return e;
    if ((e = malloc_t(m, &m->aT, (size_t)B * m->hid)) != cudaSuccess) return e;
    if ((e = malloc_t(m, &m->bT, (size_t)B * m->hid)) != cudaSuccess) return e;
    if ((e = malloc_t(m, &m->y, B)) != cudaSuccess) return e;
    if ((e = malloc_t(m, &m->dy, B)) != cudaSuccess) return e;
    if ((e = malloc_t(m, &m->part, (size_t)((B + kRowChunk - 1) / kRowChunk) * m->hid)) != cudaSuccess) return e;
    m->cap = B;
    return cudaSuccess;
}

cudaError_t forward_pass(titan_mlp *m, const __nv_bfloat16 *x, uint32_t B, float *y) {
    cudaError_t e;
    const __nv_bfloat16 *a = x;
    for (int l = 0; l < 3; ++l) {
        EpiArgs ep{EPI_BIAS_GELU, (int)m->hid, m->p + m->off_b[l], m->Z[l], m->H[l], nullptr};
        if ((e = gemm_tn(a, m->wt[l], (int)B, (int)m->hid, (int)layer_in(m, l), ep, m->stream, m->spin_limit, m->err)) != cudaSuccess)
            return e;
        a = m->H[l];
    }
    k_out_layer<<<nblk(B, 8), 256, 0, m->stream>>>(m->H[2], m->p + m->off_w4, m->p + m->off_b4, y, (int)B, (int)m->hid);
    return cudaGetLastError();
}

cudaError_t backward_pass(titan_mlp *m, const __nv_bfloat16 *x, const float *t, uint32_t B, float *loss) {
    cudaError_t e = forward_pass(m, x, B, m->y);
    if (e != cudaSuccess) return e;
    k_loss<<<1, 256, 0, m->stream>>>(m->y, t, m->dy, loss, (int)B);
    const int chunks = ((int)B + kRowChunk - 1) / kRowChunk;
    k_out_backward<<<dim3(nblk(m->hid, 128), chunks), 128, 0, m->stream>>>(m->H[2], m->Z[2], m->dy, m->p + m->off_w4,
                                                                          m->part, m->dZ[2], (int)B, (int)m->hid);
    k_col_sum_final<<<nblk(m->hid + 1, 128), 128, 0, m->stream>>>(m->part, chunks, (int)m->hid, m->g + m->off_w4,
                                                                   m->dy, (int)B, m->g + m->off_b4);
    for (int l = 2; l >= 0; --l) {
        // dW_l^T (hid x in_l) = dZ_l^T (hid x B) . A_{l-1}^T (in_l x B)^T
        const uint32_t in = layer_in(m, l);
        const __nv_bfloat16 *act = l == 0 ? x : m->H[l - 1];
        __nv_bfloat16 *actT = l == 0 ? m->xT : m->aT;
        k_transpose_bf16<<<dim3(nblk(m->hid, 32), nblk(B, 32)), dim3(32, 8), 0, m->stream>>>(m->dZ[l], m->bT, (int)B, (int)m->hid);
        k_transpose_bf16<<<dim3(nblk(in, 32), nblk(B, 32)), dim3(32, 8), 0, m->stream>>>(act, actT, (int)B, (int)in);
        EpiArgs ep{EPI_F32, (int)in, nullptr, m->g + m->off_w[l], nullptr, nullptr};
        if ((e = gemm_tn(m->bT, actT, (int)m->hid, (int)in, (int)B, ep, m->stream, m->spin_limit, m->err)) != cudaSuccess)
            return e;
        k_col_sum_part<<<dim3(nblk(m->hid, 128), chunks), 128, 0, m->stream>>>(m->dZ[l], m->part, (int)B, (int)m->hid);
        k_col_sum_final<<<nblk(m->hid, 128), 128, 0, m->stream>>>(m->part, chunks, (int)m->hid, m->g + m->off_b[l],
                                                                  nullptr, (int)B, nullptr);
        if (l > 0) {
            // dZ_{l-1} = (dZ_l . W_l^T) * GELU'(Z_{l-1}):  A = dZ_l (B x hid), B operand = W_l (in x hid)
            EpiArgs ep2{EPI_GELU_GRAD, (int)m->hid, nullptr, nullptr, m->dZ[l - 1], m->Z[l - 1]};
            if ((e = gemm_tn(m->dZ[l], m->w[l], (int)B, (int)in, (int)m->hid, ep2, m->stream, m->spin_limit, m->err)) != cudaSuccess)
                return e;
        }
    }
    return cudaGetLastError();
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

titan_status titan_gemm_bf16_tn(uint32_t M, uint32_t N, uint32_t K, const uint16_t *A_dev, const uint16_t *B_dev,
                                float *C_dev, void *stream) {
    if (!A_dev || !B_dev || !C_dev) return mfail(nullptr, TITAN_E_INVALID, "titan_gemm_bf16_tn: null pointer");
    if (M % BM || N % BN || K % BK || !M || !N || !K)
        return mfail(nullptr, TITAN_E_INVALID, "titan_gemm_bf16_tn: M and N must be multiples of 128, K of 64");
    // one device error flag per device ordinal, allocated on first use with that device current
    static int *err_of[64] = {};
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return mfail(nullptr, TITAN_E_CUDA, "titan_gemm_bf16_tn: no current device");
    int *err = nullptr;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!err_of[dev]) {
            if (cudaMalloc(&err_of[dev], sizeof(int)) != cudaSuccess)
                return mfail(nullptr, TITAN_E_OOM, "titan_gemm_bf16_tn: error flag");
            if (cudaMemset(err_of[dev], 0, sizeof(int)) != cudaSuccess)
                return mfail(nullptr, TITAN_E_CUDA, "titan_gemm_bf16_tn: error flag");
        }
        err = err_of[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    EpiArgs ep{EPI_F32, (int)N, nullptr, C_dev, nullptr, nullptr};
    cudaError_t e = gemm_tn(A_dev, B_dev, (int)M, (int)N, (int)K, ep, st, 1u << 22, err);
    if (e != cudaSuccess) return mfail(nullptr, TITAN_E_CUDA, std::string("titan_gemm_bf16_tn: ") + cudaGetErrorString(e));
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return mfail(nullptr, TITAN_E_CUDA, std::string("titan_gemm_bf16_tn: ") + cudaGetErrorString(e));
    int flag = 0;
    cudaMemcpy(&flag, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (flag) {
        cudaMemset(err, 0, sizeof(int));
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
    MLP_CK(m, ensure_batch(m, batch));
    MLP_CK(m, backward_pass(m, reinterpret_cast<const __nv_bfloat16 *>(x_dev), t_dev, batch, loss_dev));
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    ++m->adam_t;
    const float c1 = 1.f - std::pow(b1, (float)m->adam_t), c2 = 1.f - std::pow(b2, (float)m->adam_t);
    k_adam<<<nblk(m->n_params, 256), 256, 0, m->stream>>>(m->p, m->g, m->m, m->v, m->n_params, lr, b1, b2, eps, c1, c2);
    MLP_CK(m, cudaGetLastError());
    MLP_CK(m, refresh_bf16(m));
    return TITAN_OK;
}

titan_status titan_mlp_sync(titan_mlp *m) { return m ? check_err(m) : TITAN_E_INVALID; }

const char *titan_mlp_last_error(const titan_mlp *m) { return m ? m->error.c_str() : ""; }

titan_status titan_mlp_destroy(titan_mlp *m) {
    if (!m) return TITAN_OK;
    cudaStreamSynchronize(m->stream);
    for (void *p : m->allocs) cudaFree(p);
    if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
    delete m;
    return TITAN_OK;
}

}  // extern "C"
