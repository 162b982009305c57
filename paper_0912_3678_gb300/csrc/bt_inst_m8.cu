// Kernel instantiations for block order m = 8.
#include "bt_inst.cuh"
namespace bt {
const Launchers* launchers_m8() { return Inst<8>::table(); }
}  // namespace bt
