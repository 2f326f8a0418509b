// fused_kernel.cu -- dense k-qubit block on the tensor cores (placeholder:
// the tcgen05 kernel is added next; until then blocks run on the CUDA-core
// dense kernel).
#include "internal.h"

int launch_block_tc(qsim *s, const int *qubits, int k, const cd *m) {
    (void)s; (void)qubits; (void)k; (void)m;
    return QSIM_ENOTSUP;
}
