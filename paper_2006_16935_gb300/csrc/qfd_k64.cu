// complex128 instantiation of the pass kernels and launchers.
#include "qfd_launch_impl.cuh"

namespace qfd {
QFD_INSTANTIATE_LAUNCHERS(double)
}  // namespace qfd
