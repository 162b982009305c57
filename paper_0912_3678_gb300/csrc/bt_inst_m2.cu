// Kernel instantiations for block order m = 2.
#include "bt_inst.cuh"
namespace bt {
const Launchers* launchers_m2() { return Inst<2>::table(); }
}  // namespace bt
