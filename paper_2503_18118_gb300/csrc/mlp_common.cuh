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

// Packed inference image: the three 256 x 256 layers as BF16 tiles of the
// tensor-core B operand (output unit = row, input = K, 128-byte swizzle), one
// 16 KB tile per (layer, output half, 64-input chunk), then the FP32 parts.
constexpr int MLP_TILE_BYTES = 128 * 64 * 2;
constexpr int MLP_TILES = 3 * 2 * 4;
constexpr int64_t MLP_PK_F32 = (int64_t)MLP_TILES * MLP_TILE_BYTES;  // byte offset of the FP32 block
// floats of the FP32 block: W0 [6][256], b0, b1, b2, b3 [256], W4 [256][2], b4 [2]
constexpr int MLP_PK_W0 = 0, MLP_PK_B0 = 1536, MLP_PK_B1 = 1792, MLP_PK_B2 = 2048, MLP_PK_B3 = 2304,
              MLP_PK_W4 = 2560, MLP_PK_B4 = 3072, MLP_PK_NF = 3074;
static_assert(MLP_PK_F32 + MLP_PK_NF * 4 <= XLMIMO_MLP_PACKED_BYTES, "packed image size");

// Byte offset, inside its 16 KB tile, of row r (0..127), column c (0..63):
// 8-row groups 1024 B apart, 128 B per row, 16-byte units XOR-swizzled by r % 8.
__host__ __device__ __forceinline__ int sw128_offset(int r, int c) {
    return (r >> 3) * 1024 + (r & 7) * 128 + ((((c >> 3) ^ (r & 7)) & 7) << 4) + (c & 7) * 2;
}

// Row q of a trial's pair list -> users (i, j), i < j, pairs in row order.
__device__ __forceinline__ void pair_index(int q, int K, int& i, int& j) {
    int ii = 0, rl = K - 1;
    while (q >= rl && rl > 0) { q -= rl; ++ii; --rl; }
    i = ii;
    j = ii + 1 + q;
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

}  // namespace xl
