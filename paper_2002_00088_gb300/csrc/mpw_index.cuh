// mpw_index.cuh -- index walks of the ghost-fill kernels: the points of a
// hollow box (the outer ghost shell of a patch) and the elements of a
// two-field block visited with a fixed thread stride.
//
// The file includes nothing: the CUDA qualifiers and max() it names come
// from the translation units that include it.
#pragma once

namespace mpw {

// Position of element e of a [2][d2][d1][d0] block (x fastest, then y, z,
// field) and its advance by STRIDE threads: the divisions are taken once per
// thread, every later step is a mixed-radix addition with single carries
// (each digit and its increment are below the radix).
template <int STRIDE>
struct BlockWalk {
  int o0, o1, o2, f;
  int a0, a1, a2, a3;
  int d0, d1, d2;
  __device__ __forceinline__ BlockWalk(int e, int d0_, int d1_, int d2_) : d0(d0_), d1(d1_), d2(d2_) {
    int q = e / d0;
    o0 = e - q * d0;
    o1 = q % d1;
    q /= d1;
    o2 = q % d2;
    f = q / d2;
    q = STRIDE / d0;
    a0 = STRIDE - q * d0;
    a1 = q % d1;
    q /= d1;
    a2 = q % d2;
    a3 = q / d2;
  }
  __device__ __forceinline__ void next() {
    o0 += a0;
    int c = o0 >= d0;
    o0 -= c ? d0 : 0;
    o1 += a1 + c;
    c = o1 >= d1;
    o1 -= c ? d1 : 0;
    o2 += a2 + c;
    c = o2 >= d2;
    o2 -= c ? d2 : 0;
    f += a3 + c;
  }
};

// Maps idx in [0, Ox*Oy*Oz - Ix*Iy*Iz) onto the points of the hollow box of
// outer extent O whose walls are th thick (I = max(O - 2 th, 0)).
// IdxT is the index type: unsigned (32-bit divisions, several times cheaper on
// the GPU) when the shell holds fewer than 2^31 points, whose products
// below then fit as well; long long otherwise.
template <typename IdxT>
__device__ __forceinline__ void shell_point_t(IdxT idx, const int O[3], int th, int& x, int& y, int& z) {
  const int Ix = max(O[0] - 2 * th, 0), Iy = max(O[1] - 2 * th, 0), Iz = max(O[2] - 2 * th, 0);
  const IdxT pxy = (IdxT)O[0] * (IdxT)O[1];
  const IdxT nz = pxy * (IdxT)(O[2] - Iz);
  if (idx < nz) {
    const int zs = (int)(idx / pxy);
    const IdxT r = idx - (IdxT)zs * pxy;
    z = zs < th ? zs : zs + Iz;
    y = (int)(r / (IdxT)O[0]);
    x = (int)(r - (IdxT)y * (IdxT)O[0]);
    return;
  }
  idx -= nz;
  const IdxT rowsy = (IdxT)O[0] * (IdxT)(O[1] - Iy);
  const IdxT ny = rowsy * (IdxT)Iz;
  if (idx < ny) {
    const int zz = (int)(idx / rowsy);
    const IdxT r = idx - (IdxT)zz * rowsy;
    z = th + zz;
    const int ys = (int)(r / (IdxT)O[0]);
    x = (int)(r - (IdxT)ys * (IdxT)O[0]);
    y = ys < th ? ys : ys + Iy;
    return;
  }
  idx -= ny;
  const int wx = O[0] - Ix;
  const IdxT per_z = (IdxT)wx * (IdxT)Iy;
  const int zz = (int)(idx / per_z);
  const IdxT r = idx - (IdxT)zz * per_z;
  z = th + zz;
  const int yy = (int)(r / (IdxT)wx);
  const int xs = (int)(r - (IdxT)yy * (IdxT)wx);
  y = th + yy;
  x = xs < th ? xs : xs + Ix;
}

__device__ __forceinline__ void shell_point(long long idx, const int O[3], int th, int& x, int& y, int& z) {
  shell_point_t<long long>(idx, O, th, x, y, z);
}

}  // namespace mpw
