// Kernel instantiations for block order m = 1.
#include "bt_inst.cuh"
namespace bt {
const Launchers* launchers_m1() { return Inst<1>::table(); }
}  // namespace bt
