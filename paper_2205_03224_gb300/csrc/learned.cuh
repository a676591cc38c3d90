// Learned interface correction (not in the paper): a 4-layer 27-tap (3x3x3)
// convolutional network over the unknowns of the deepest Schur level's
// interface, trained on (rho, S_hat^{-1} rho) pairs the method generates and
// applied inside M^{-1} as
//     rho = z2 - S_hat y2,  S_hat = C - E (U^{-1} L^{-1}) F  (level l* = nlev-2)
//     y2 <- y2 + (||rho|| / d) * net(rho / ||rho||)
// with d the mean |diagonal| of S_hat.  Weights are BF16 with FP32 master
// copies (Adam); all arithmetic accumulates in FP32.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>

namespace gemslr {

constexpr int kNetLayers = 4;

struct NetDev {
    int S = 0, C = 0;                 // sites, hidden channels
    int cin[kNetLayers], cout[kNetLayers];
    int32_t *nbr = nullptr;           // S x 27 (site index or -1)
    int32_t *nbr_t = nullptr;         // S x 27 transposed taps: site u's partner for tap t is nbr[u][26-t]
    float *W[kNetLayers], *b[kNetLayers];          // FP32 master
    __nv_bfloat16 *Wb[kNetLayers];                 // BF16 copies used by every pass
    float *gW[kNetLayers], *gb[kNetLayers];        // gradients
    float *mW[kNetLayers], *vW[kNetLayers], *mb[kNetLayers], *vb[kNetLayers];   // Adam moments
    double dscale = 1.0;              // mean |diag S_hat|
    int64_t nparams = 0;
    int adam_t = 0;
};

// Buffers of the in-apply stage.
template <typename VT>
struct LearnedStage {
    bool enabled = false;
    NetDev *net = nullptr;
    VT *zsave = nullptr;              // z2 of level l* (S values)
    VT *work2 = nullptr;              // n-length scratch for S_hat y2
    const double *zeros = nullptr;    // n zeros
    const int64_t *C_rp = nullptr;    // full C of level l* (S x S), tail-local columns
    const int32_t *C_ci = nullptr;
    const VT *C_v = nullptr;
    float *act0 = nullptr, *act1 = nullptr, *act2 = nullptr;   // S x C activations (N = 1)
    float *rnorm = nullptr;           // ||rho|| of the current application
};

}  // namespace gemslr
