// krylov_f64.cu -- FP64 storage and arithmetic (plain BiCGStab, the outer
// true residual, odd-site reconstruction for the force).
#include "krylov_impl.cuh"

namespace sf {
const KrylovOps& ops_f64() {
    static const KrylovOps t = OpsImpl<P64, P64>::table(Prec::F64, Prec::F64);
    return t;
}
}  // namespace sf
