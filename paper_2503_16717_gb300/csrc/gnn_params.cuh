// Parameter layout of the learned-SPAI network (3 message-passing layers of width 32),
// shared by its kernels and its host side.  One flat float32 vector theta (and its
// bfloat16 copy used by the forward kernels):
//   [Wn 32x2 | bn 32 | We 32x3 | be 32 | layer 0 | layer 1 | layer 2 | wo 96 | bo 1]
//   layer l: [Wm 32x64 | bm 32 | Wh 32x64 | bh 32], every matrix row-major (output c,
//   input k): Wm's inputs are [e_ij ; h_j], Wh's inputs are [h_i ; agg_i].
#pragma once

namespace rbo {
namespace gnn {

constexpr int W = 32;
constexpr int NL = 3;
constexpr int OFF_WN = 0, OFF_BN = 64, OFF_WE = 96, OFF_BE = 192, OFF_L0 = 224;
constexpr int LAYER_SZ = 2048 + 32 + 2048 + 32;
constexpr int OFF_WO = OFF_L0 + NL * LAYER_SZ;  // 12704
constexpr int OFF_BO = OFF_WO + 96;
constexpr int NPARAM = OFF_BO + 1;               // 12801
__host__ __device__ constexpr int off_wm(int l) { return OFF_L0 + l * LAYER_SZ; }
__host__ __device__ constexpr int off_bm(int l) { return off_wm(l) + 2048; }
__host__ __device__ constexpr int off_wh(int l) { return off_wm(l) + 2080; }
__host__ __device__ constexpr int off_bh(int l) { return off_wm(l) + 4128; }

}  // namespace gnn
}  // namespace rbo
