// Kernel instantiations for block order m = 32.
#include "bt_inst.cuh"
namespace bt {
const Launchers* launchers_m32() { return Inst<32>::table(); }
}  // namespace bt
