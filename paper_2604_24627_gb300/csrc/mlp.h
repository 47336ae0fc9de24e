// The surrogate MLP on the GPU (internal to libaxpic).
#pragma once
#include <cuda_runtime.h>

namespace axpic {

// Parameter layout (FP32): W1[4][64], b1[64], W2[64][64], b2[64], W3[64][96], b3[96].
constexpr int kOffW1 = 0, kOffB1 = 256, kOffW2 = 320, kOffB2 = 4416, kOffW3 = 4480, kOffB3 = 10624;
constexpr int kMlpParams = 10720;

struct Mlp {
  cudaStream_t st = nullptr;
  float *P = nullptr, *G = nullptr, *Ma = nullptr, *Va = nullptr;  // params, grads, Adam moments
  float *h1 = nullptr, *h2 = nullptr, *z = nullptr, *dz = nullptr, *dh = nullptr;
  float* part = nullptr;  // split-K partials of the weight gradients
  int* err = nullptr;
  double* loss = nullptr;
  int cap = 0;
  long t = 0;  // Adam steps taken

  ~Mlp();
  cudaError_t init(cudaStream_t s);
  cudaError_t reserve(int n);
  // z[n][96] = network(X[n][4]) (normalised outputs); out NULL: the own
  // buffer z, taken after the work buffers are reserved for n rows (never
  // pass z itself: reserving may reallocate it)
  cudaError_t forward(const float* X, int n, float* out);
  // G = d loss / d P and *loss, loss = sum (z - Zt)^2 / n
  cudaError_t gradients(const float* X, const float* Zt, int n);
  cudaError_t adam(float lr);
  const float* W1() const { return P + kOffW1; }
  const float* b1() const { return P + kOffB1; }
  const float* W2() const { return P + kOffW2; }
  const float* b2() const { return P + kOffB2; }
  const float* W3() const { return P + kOffW3; }
  const float* b3() const { return P + kOffB3; }
};

}  // namespace axpic
