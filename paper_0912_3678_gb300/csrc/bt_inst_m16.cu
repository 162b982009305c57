// Kernel instantiations for block order m = 16.
#include "bt_inst.cuh"
namespace bt {
const Launchers* launchers_m16() { return Inst<16>::table(); }
}  // namespace bt
