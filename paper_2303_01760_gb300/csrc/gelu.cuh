// GELU of the learned predictor's fused tensor-core pass, shared with the
// elementwise evaluator that pins it (probe.cu).
#pragma once

// erf(x) for x >= 0 by Abramowitz and Stegun 7.1.28:
//   erf(x) = 1 - (1 + a1 x + a2 x^2 + ... + a6 x^6)^-16,
// |error| <= 3e-7 in exact arithmetic.  In FP32 the Horner sum (positive
// terms, relative error <= 6 u) and the reciprocal (<= 2 ulp) reach the
// sixteenth power with their relative error multiplied by 16, so the
// evaluated t = (...)^-16 carries a relative error below 9e-6 and
// |erf_as(x) - erf(x)| <= 3e-7 + 9e-6 (1 - erf(x)) + 2^-24 -- far below the
// bf16 rounding (2^-9) of the activations it feeds.  One reciprocal is the
// only special function.
__device__ __forceinline__ float erf_as(float x) {
  float p = fmaf(x, 0.0000430638f, 0.0002765672f);
  p = fmaf(x, p, 0.0001520143f);
  p = fmaf(x, p, 0.0092705272f);
  p = fmaf(x, p, 0.0422820123f);
  p = fmaf(x, p, 0.0705230784f);
  p = fmaf(x, p, 1.0f);
  float t = __fdividef(1.0f, p);  // (1 + ...)^-1, then ^16 by squaring
  t *= t;
  t *= t;
  t *= t;
  t *= t;
  return 1.0f - t;
}

// GELU(z) = z Phi(z) = (z + |z| erf(|z| / sqrt 2)) / 2.
__device__ __forceinline__ float gelu(float z) {
  return 0.5f * fmaf(fabsf(z), erf_as(fabsf(z) * 0.70710678118654752f), z);
}
