// Interpolation weights of one coordinate, the scheme D-SKI differentiates
// (Sec. 3.1): for grid parameter t = (x - lo)/h, cell c = floor(t) and
// fraction f = t - c in [0, 1), the S stencil nodes c - S/2 + 1 + o
// (o = 0..S-1) get weight phi(t - node) and derivative weight
// phi'(t - node) / h (the caller multiplies by 1/h).
//
// S = 4: Keys' cubic convolution kernel (a = -1/2),
//   phi(s) = 3/2|s|^3 - 5/2|s|^2 + 1           for |s| <= 1,
//   phi(s) = -1/2|s|^3 + 5/2|s|^2 - 4|s| + 2   for 1 < |s| < 2.
// S = 6: the six-point quintic kernel the paper uses (Meijering et al.,
//   1999): even, piecewise quintic on the knots 0..3, interpolating, C^3
//   across the knots and at |s| = 3, reproducing quadratics (free parameter
//   3/64).  With u the distance past the piece's left knot:
//   |s| in [0, 1]: 1 - 17/8 s^2 + 63/32 s^4 - 27/32 s^5       (s = |s|)
//   |s| in [1, 2]: u (-19/32 + 5/4 u - 9/16 u^2 - 19/64 u^3 + 13/64 u^4)
//   |s| in [2, 3]: 3/64 u (1 - u)^4.
// Each branch below is that polynomial at the node's known piece and sign
// (factored for the cubic, Horner form for the quintic).
#pragma once

namespace dski {

// With g = 1 - f the four pieces factor (expand to check against phi):
//   node c-1 (s = 1 + f):  phi = -f g^2 / 2,          phi' = g (f - g / 2)
//   node c   (s = f):      phi = 1 + f^2 (3f/2 - 5/2), phi' = f (9f/2 - 5)
//   node c+1 (s = -g):     phi = 1 + g^2 (3g/2 - 5/2), phi' = -g (9g/2 - 5)
//   node c+2 (s = -1 - g): phi = -g f^2 / 2,          phi' = f (f / 2 - g)
// (shared powers: ~21 operations for the eight values).
template <class T>
__device__ __forceinline__ void keys4(T f, T w[4], T dw[4]) {
  const T g = T(1) - f;
  const T f2 = f * f, g2 = g * g;
  w[0] = (T(-0.5) * f) * g2;
  w[1] = fma(f2, fma(T(1.5), f, T(-2.5)), T(1));
  w[2] = fma(g2, fma(T(1.5), g, T(-2.5)), T(1));
  w[3] = (T(-0.5) * g) * f2;
  dw[0] = g * fma(T(-0.5), g, f);
  dw[1] = f * fma(T(4.5), f, T(-5));
  dw[2] = g * fma(T(-4.5), g, T(5));
  dw[3] = f * fma(T(0.5), f, -g);
}

// quintic pieces and their derivatives (argument: |s| for the inner piece,
// u in [0, 1] for the others)
template <class T>
__device__ __forceinline__ T q5_in(T s) {
  const T s2 = s * s;
  return (((T(-27.0 / 32.0) * s + T(63.0 / 32.0)) * s2) + T(-17.0 / 8.0)) * s2 + T(1);
}
template <class T>
__device__ __forceinline__ T q5_in_d(T s) {
  const T s2 = s * s;
  return ((T(-135.0 / 32.0) * s + T(63.0 / 8.0)) * s2 + T(-17.0 / 4.0)) * s;
}
template <class T>
__device__ __forceinline__ T q5_mid(T u) {
  return ((((T(13.0 / 64.0) * u + T(-19.0 / 64.0)) * u + T(-9.0 / 16.0)) * u + T(5.0 / 4.0)) * u +
          T(-19.0 / 32.0)) * u;
}
template <class T>
__device__ __forceinline__ T q5_mid_d(T u) {
  return (((T(65.0 / 64.0) * u + T(-19.0 / 16.0)) * u + T(-27.0 / 16.0)) * u + T(5.0 / 2.0)) * u +
         T(-19.0 / 32.0);
}
template <class T>
__device__ __forceinline__ T q5_out(T u) {
  const T v = T(1) - u, v2 = v * v;
  return T(3.0 / 64.0) * u * (v2 * v2);
}
template <class T>
__device__ __forceinline__ T q5_out_d(T u) {
  const T v = T(1) - u;
  return T(3.0 / 64.0) * (v * v * v) * (T(1) - T(5) * u);
}

template <class T>
__device__ __forceinline__ void quintic6(T f, T w[6], T dw[6]) {
  const T g = T(1) - f;
  w[0] = q5_out(f);   // node c-2: s = 2 + f
  dw[0] = q5_out_d(f);
  w[1] = q5_mid(f);   // node c-1: s = 1 + f
  dw[1] = q5_mid_d(f);
  w[2] = q5_in(f);    // node c  : s = f
  dw[2] = q5_in_d(f);
  w[3] = q5_in(g);    // node c+1: s = -(1 - f)
  dw[3] = -q5_in_d(g);
  w[4] = q5_mid(g);   // node c+2: s = -(2 - f)
  dw[4] = -q5_mid_d(g);
  w[5] = q5_out(g);   // node c+3: s = -(3 - f)
  dw[5] = -q5_out_d(g);
}

// All S weights and derivative weights (derivatives w.r.t. t).
template <int S, class T>
__device__ __forceinline__ void stencil_weights(T f, T* w, T* dw) {
  static_assert(S == 4 || S == 6, "stencil of 4 (cubic) or 6 (quintic) nodes");
  if constexpr (S == 4) keys4<T>(f, w, dw);
  else quintic6<T>(f, w, dw);
}

}  // namespace dski
