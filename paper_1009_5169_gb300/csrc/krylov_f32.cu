// krylov_f32.cu -- FP32 storage and arithmetic (inner solver under FP64
// defect correction).
#include "krylov_impl.cuh"

namespace sf {
const KrylovOps& ops_f32() {
    static const KrylovOps t = OpsImpl<P32, P32>::table(Prec::F32, Prec::F32);
    return t;
}
}  // namespace sf
