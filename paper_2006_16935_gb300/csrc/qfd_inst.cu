// One (arithmetic policy, lattice size) instantiation of the pass launchers.
// The build compiles this file once per pair, with -DQFD_POLICY=F64|F32|DF and
// -DQFD_N=8..1024, so that the unrolled kernels compile in parallel.
#include "qfd_launch_impl.cuh"

#if !defined(QFD_POLICY) || !defined(QFD_N)
#error "compile with -DQFD_POLICY=<F64|F32|DF> -DQFD_N=<lattice size>"
#endif

namespace qfd {
template struct Launch<QFD_POLICY, QFD_N>;
}  // namespace qfd
