// Parameter layout of the troubled-cell indicator network and the forward
// entry used by the gated residual.  Flat FP32 parameter vector, in order:
// W1 [64][32], b1 [64], W2 [64][64], b2 [64], w3 [64], b3 [1].
#pragma once

#include <cstdint>

struct ucns_mlp;

namespace ucnsnet {
constexpr int kOffW1 = 0, kOffB1 = 2048, kOffW2 = 2112, kOffB2 = 6208, kOffW3 = 6272, kOffB3 = 6336;
constexpr int kParams = 6337;
constexpr int kFeatures = 32;
// logits z (optional), flags z > threshold (optional) and the BF16 first
// hidden layer h1 [n][64] (optional) of n BF16 feature rows
int forward(ucns_mlp* m, const void* X, int64_t n, float* z, uint8_t* flag, float threshold, void* stream,
            void* h1 = nullptr);
}  // namespace ucnsnet
