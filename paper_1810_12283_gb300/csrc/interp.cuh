// Keys cubic-convolution weights (a = -1/2), the interpolation scheme D-SKI
// differentiates (Sec. 3.1).  For one coordinate with grid parameter
// t = (x - lo)/h, cell c = floor(t) and fraction f = t - c in [0, 1), the
// four stencil nodes c-1+o (o = 0..3) get weight omega(f + 1 - o) and
// derivative weight omega'(f + 1 - o) / h, where
//   omega(s) = 3/2|s|^3 - 5/2|s|^2 + 1           for |s| <= 1,
//   omega(s) = -1/2|s|^3 + 5/2|s|^2 - 4|s| + 2   for 1 < |s| < 2,
// (Keys' kernel with a = -1/2) and omega' its derivative in s.  Each branch
// below is that polynomial at the node's known sign/branch, in Horner form.
#pragma once

namespace dski {

// All four weights and derivative weights (derivatives w.r.t. t; the caller
// multiplies by 1/h).
template <class T>
__device__ __forceinline__ void keys4(T f, T w[4], T dw[4]) {
  const T s0 = f + T(1);   // node c-1: s in [1, 2)
  const T s1 = f;          // node c  : s in [0, 1)
  const T s2 = T(1) - f;   // node c+1: |s| in (0, 1], s <= 0
  const T s3 = T(2) - f;   // node c+2: |s| in (1, 2], s <= -1
  w[0] = ((T(-0.5) * s0 + T(2.5)) * s0 - T(4)) * s0 + T(2);
  w[1] = (T(1.5) * s1 - T(2.5)) * s1 * s1 + T(1);
  w[2] = (T(1.5) * s2 - T(2.5)) * s2 * s2 + T(1);
  w[3] = ((T(-0.5) * s3 + T(2.5)) * s3 - T(4)) * s3 + T(2);
  dw[0] = (T(-1.5) * s0 + T(5)) * s0 - T(4);
  dw[1] = (T(4.5) * s1 - T(5)) * s1;
  dw[2] = -((T(4.5) * s2 - T(5)) * s2);
  dw[3] = -((T(-1.5) * s3 + T(5)) * s3 - T(4));
}

// Weight and derivative weight of the single node c-1+o.
template <class T>
__device__ __forceinline__ void keys1(T f, int o, T& w, T& dw) {
  switch (o) {
    case 0: {
      const T s = f + T(1);
      w = ((T(-0.5) * s + T(2.5)) * s - T(4)) * s + T(2);
      dw = (T(-1.5) * s + T(5)) * s - T(4);
    } break;
    case 1: {
      const T s = f;
      w = (T(1.5) * s - T(2.5)) * s * s + T(1);
      dw = (T(4.5) * s - T(5)) * s;
    } break;
    case 2: {
      const T s = T(1) - f;
      w = (T(1.5) * s - T(2.5)) * s * s + T(1);
      dw = -((T(4.5) * s - T(5)) * s);
    } break;
    default: {
      const T s = T(2) - f;
      w = ((T(-0.5) * s + T(2.5)) * s - T(4)) * s + T(2);
      dw = -((T(-1.5) * s + T(5)) * s - T(4));
    } break;
  }
}

}  // namespace dski
