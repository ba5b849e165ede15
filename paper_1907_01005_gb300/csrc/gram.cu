// Block-sparse Gram products C = A^T B over stored blocks (Alg. 8).
//
// Work is organised by output block: an item is a run of row blocks that all
// hold both column blocks (c1, c2); its CTA accumulates the w1 x w2 block
// C[c1, c2] over those row blocks in FP64 and adds it into the dense FP64
// result.  For the Euclidean P^T P only pairs c1 <= c2 are listed and the
// result is mirrored.
#include "fe_internal.h"

namespace femf {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) gram_pairs_kernel(const GramArgs<T> g) {
    const GramItem it = g.items[blockIdx.x];
    const int c1 = it.c1, c2 = it.c2;
    const int col1 = g.cb_ptr[c1], col2 = g.cb_ptr[c2];
    const int w1 = g.cb_ptr[c1 + 1] - col1, w2 = g.cb_ptr[c2 + 1] - col2;
    const int a = threadIdx.x / kMaxW, b = threadIdx.x % kMaxW;
    if (a >= w1 || b >= w2) return;
    const int ld1 = g.ld[c1], ld2 = g.ld[c2];
    double acc = 0.0;
    for (int e = it.begin; e < it.end; ++e) {
        const GramEntry en = g.entries[e];
        const T* pa = g.A + en.offA + a;
        const T* pb = g.B + en.offB + b;
        for (int r = 0; r < en.rows; ++r)
            acc = fma(static_cast<double>(pa[(int64_t)r * ld1]), static_cast<double>(pb[(int64_t)r * ld2]), acc);
    }
    atomicAdd(&g.G[(int64_t)(col1 + a) * g.n_cols + col2 + b], acc);
    if (g.symmetric && c1 != c2) atomicAdd(&g.G[(int64_t)(col2 + b) * g.n_cols + col1 + a], acc);
}

}  // namespace

template <typename T>
cudaError_t launch_gram(const GramArgs<T>& g, cudaStream_t s) {
    if (g.n_items == 0) return cudaSuccess;
    gram_pairs_kernel<T><<<(unsigned)g.n_items, kMaxW * kMaxW, 0, s>>>(g);
    return cudaGetLastError();
}

template cudaError_t launch_gram<float>(const GramArgs<float>&, cudaStream_t);
template cudaError_t launch_gram<double>(const GramArgs<double>&, cudaStream_t);

}  // namespace femf
