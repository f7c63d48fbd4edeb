// Shapes, parameter layout and per-pair features of the correlation
// surrogate, shared by the training kernels (mlp.cu) and the tensor-core
// inference kernel (mlp_tc.cu).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace xl {

constexpr int MLP_IN = XLMIMO_MLP_IN;
constexpr int MLP_W = XLMIMO_MLP_WIDTH;
constexpr int MLP_OUT = XLMIMO_MLP_OUT;
constexpr int MLP_LAYERS = XLMIMO_MLP_HIDDEN + 1;  // linear layers

__host__ __device__ constexpr int mlp_in(int l) { return l == 0 ? MLP_IN : MLP_W; }
__host__ __device__ constexpr int mlp_out(int l) { return l == MLP_LAYERS - 1 ? MLP_OUT : MLP_W; }
// first float of layer l's W [in][out] (its bias [out] follows W)
__host__ __device__ constexpr int64_t mlp_off(int l) {
    return l == 0 ? 0 : mlp_off(l - 1) + (int64_t)(mlp_in(l - 1) + 1) * mlp_out(l - 1);
}
static_assert(mlp_off(MLP_LAYERS) == XLMIMO_MLP_PARAMS, "parameter count");

// Packed inference image.  BF16 tiles of the tensor-core B operand (output
// unit = row, input = K, 128-byte swizzle), 16 KB each (128 output units x 64
// inputs), in the order the inference kernel consumes them:
//   tiles 0, 1     layer 0 (6 -> 256), output halves 0 and 1: inputs 0-5 hold
//                  hi(W0/2), 6-11 hi(W0/2) again, 12-17 lo(W0/2), the rest 0,
//                  to meet the A row [hi(f), lo(f), hi(f)] of the features
//                  (three BF16 products recover the FP32 sum to ~2^-16);
//   tiles 2 + 8 (l-1) + 4 h + c   layer l = 1..3, output half h, inputs 64c..64c+63,
//                  holding W_l / 2;
// then the FP32 block: b0/2, b1/2, b2/2, b3/2, W4 [256][2], b4 [2].
// Halving the weights and biases of the hidden layers (exact in BF16 and
// FP32) makes the accumulators hold z/2, the argument of the tanh form of
// SiLU, silu(z) = z/2 (1 + tanh(z/2)).
constexpr int MLP_TILE_BYTES = 128 * 64 * 2;
constexpr int MLP_TILES = 2 + 3 * 2 * 4;
constexpr int64_t MLP_PK_F32 = (int64_t)MLP_TILES * MLP_TILE_BYTES;  // byte offset of the FP32 block
constexpr int MLP_PK_B0 = 0, MLP_PK_B1 = 256, MLP_PK_B2 = 512, MLP_PK_B3 = 768, MLP_PK_W4 = 1024,
              MLP_PK_B4 = 1536, MLP_PK_NF = 1538;
static_assert(MLP_PK_F32 + MLP_PK_NF * 4 <= XLMIMO_MLP_PACKED_BYTES, "packed image size");

// Byte offset, inside its 16 KB tile, of row r (0..127), column c (0..63):
// 8-row groups 1024 B apart, 128 B per row, 16-byte units XOR-swizzled by r % 8.
__host__ __device__ __forceinline__ int sw128_offset(int r, int c) {
    return (r >> 3) * 1024 + (r & 7) * 128 + ((((c >> 3) ^ (r & 7)) & 7) << 4) + (c & 7) * 2;
}

// Row q of a trial's pair list -> users (i, j), i < j, pairs in row order.
// Row i starts at S(i) = i (2K - 1 - i) / 2; the FP32 root of S(i) = q gives i
// to within one, which the two loops correct.
__device__ __forceinline__ void pair_index(int q, int K, int& i, int& j) {
    const float a = (float)(2 * K - 1);
    int ii = (int)((a - sqrtf(fmaxf(a * a - 8.0f * (float)q, 0.0f))) * 0.5f);
    ii = max(0, min(ii, K - 2));
    while (ii < K - 2 && ((ii + 1) * (2 * K - 2 - ii)) / 2 <= q) ++ii;
    while (ii > 0 && (ii * (2 * K - 1 - ii)) / 2 > q) --ii;
    i = ii;
    j = q - (ii * (2 * K - 1 - ii)) / 2 + ii + 1;
}

// Geometry constants of the features that do not depend on the pair.
struct FeatConst {
    float inv_lambda;
    float f_logn;    // (log2 N - 14) / 4
    float f_spacing; // (spacing / lambda - 0.5) * 4
};

inline FeatConst make_feat_const(const Geom& g) {
    FeatConst f;
    f.inv_lambda = (float)g.inv_lambda;
    f.f_logn = (float)((log2((double)g.N) - 14.0) / 4.0);
    f.f_spacing = (float)((g.spacing * g.inv_lambda - 0.5) * 4.0);
    return f;
}

// The six features of a pair, in FP32: per user (ln(r/lambda) - 7.5) / 2 and
// theta / (pi/3), theta the angle from broadside; then the array's two.
__device__ __forceinline__ void pair_features_dev(const FeatConst& fc, double xi, double yi, double xj, double yj,
                                                  float* f) {
    const float inv_third_pi = 0.954929658551372f;  // 3 / pi
    const float fxi = (float)xi, fyi = (float)yi, fxj = (float)xj, fyj = (float)yj;
    f[0] = (logf(sqrtf(fxi * fxi + fyi * fyi) * fc.inv_lambda) - 7.5f) * 0.5f;
    f[1] = atan2f(fyi, fxi) * inv_third_pi;
    f[2] = (logf(sqrtf(fxj * fxj + fyj * fyj) * fc.inv_lambda) - 7.5f) * 0.5f;
    f[3] = atan2f(fyj, fxj) * inv_third_pi;
    f[4] = fc.f_logn;
    f[5] = fc.f_spacing;
}

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// SiLU and its derivative as the training kernels evaluate them (FP32).
__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float silu_grad_f(float z) {
    const float s = 1.0f / (1.0f + expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// ---- tensor-core training GEMMs of the three 256 x 256 layers (mlp_train_tc.cu)
// Packed weights of one layer: the forward operand (output unit = row,
// input = K) then the input-gradient operand (input unit = row, output = K),
// each 4 tiles of 256 rows x 64 K (BF16, 128-byte swizzle, 32 KB).
constexpr int MT_B_TILE_BYTES = 256 * 64 * 2;
constexpr int64_t MT_PACK_LAYER_BYTES = 2LL * 4 * MT_B_TILE_BYTES;
constexpr int64_t MT_PACK_BYTES = 3 * MT_PACK_LAYER_BYTES;  // layers 1..3
// round(W_l) of layers 1..3 into `wpk` (MT_PACK_BYTES, 16-byte aligned).
int mlp_tc_pack(const float* params, unsigned char* wpk, cudaStream_t st);
// Z = round(H) round(W_l) + b, C = silu(Z) (Z may be NULL): H, Z, C [M][256].
int mlp_tc_forward(const float* h, const unsigned char* wpk, int l, const float* bias, float* z, float* c, int M,
                   cudaStream_t st);
// dZ = (G round(W_l)^T) silu'(Z_below): G, Z_below, dZ [M][256].
int mlp_tc_input_grad(const float* g, const unsigned char* wpk, int l, const float* zprev, float* dz, int M,
                      cudaStream_t st);
// part[s][0..255][256] = round(H_s)^T G_s and part[s][256][256] = the column
// sums of G_s, for slices s of k_slice rows (a multiple of 64): the weight and
// bias gradient partials of a 256 x 256 layer, rows of `part` 257 per slice.
constexpr int MT_DW_SLICE = 256;  // batch rows per weight-gradient slice of these layers
int mlp_tc_weight_grad(const float* h, const float* g, int M, int k_slice, float* part, cudaStream_t st);

}  // namespace xl
