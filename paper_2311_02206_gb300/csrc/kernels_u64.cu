// 64-bit code instantiation of every templated kernel launcher.
#include "kernels_impl.cuh"
namespace hisa {
HISA_INSTANTIATE(uint64_t)
}
