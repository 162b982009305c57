// Kernel instantiations for block order m = 4.
#include "bt_inst.cuh"
namespace bt {
const Launchers* launchers_m4() { return Inst<4>::table(); }
}  // namespace bt
