// Gram-Schmidt / parity launchers for every arithmetic policy.
#include "qfd_kernels.cuh"
#include "qfd_launch.h"

namespace qfd {

template <class A>
cudaError_t launch_gs_dots(const void* psi, const void* lower, int k, int parity, int offgrid, int64_t n, double* part,
                           int nblocks, cudaStream_t st) {
  using C = typename A::C;
  k_gs_dots<A><<<nblocks, 256, 0, st>>>((const C*)psi, (const C*)lower, k, parity, offgrid, n, part);
  return cudaGetLastError();
}

template <class A>
cudaError_t launch_gs_apply(const void* psi, const void* lower, const double* sums, int k, int parity, int offgrid,
                            int64_t n, void* out, const double* V, double* part, int check, int nblocks,
                            cudaStream_t st) {
  using C = typename A::C;
  k_gs_apply<A><<<nblocks, 256, 0, st>>>((const C*)psi, (const C*)lower, sums, k, parity, offgrid, n, (C*)out, V,
                                         part, check);
  return cudaGetLastError();
}

#define QFD_INSTANTIATE_GS(A)                                                                                     \
  template cudaError_t launch_gs_dots<A>(const void*, const void*, int, int, int, int64_t, double*, int,          \
                                         cudaStream_t);                                                           \
  template cudaError_t launch_gs_apply<A>(const void*, const void*, const double*, int, int, int, int64_t, void*, \
                                          const double*, double*, int, int, cudaStream_t);
QFD_INSTANTIATE_GS(F64)
QFD_INSTANTIATE_GS(F32)
QFD_INSTANTIATE_GS(DF)

}  // namespace qfd
