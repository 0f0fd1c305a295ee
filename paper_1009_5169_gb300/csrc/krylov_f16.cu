// krylov_f16.cu -- FP32 Krylov vectors with FP16 hop operands (per-site
// scaled spinors, FP16 links, FP32 arithmetic) under FP64 defect correction.
#include "krylov_impl.cuh"

namespace sf {
const KrylovOps& ops_f32h16() {
    static const KrylovOps t = OpsImpl<P32, P16>::table(Prec::F32, Prec::F16);
    return t;
}
}  // namespace sf
