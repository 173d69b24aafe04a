// SAMPLES packing (placeholder until the multi-sample kernels land).
#include "qisg_internal.cuh"

namespace qisg {
static int nyi() { return fail(QISG_EINVAL, "SAMPLES packing not built yet"); }
int samples_init(qisg_handle *) { return nyi(); }
int samples_half_sweep(qisg_handle *, int, int) { return nyi(); }
int samples_pt(qisg_handle *, int) { return nyi(); }
int samples_measure(qisg_handle *, int) { return nyi(); }
int samples_energies_by_slot(qisg_handle *) { return nyi(); }
int samples_get_spins(qisg_handle *, int64_t, int64_t, int8_t *) { return nyi(); }
int samples_set_spins(qisg_handle *, const int8_t *) { return nyi(); }
int samples_get_couplings(qisg_handle *, int64_t, int64_t, int8_t *) { return nyi(); }
int samples_set_couplings(qisg_handle *, const int8_t *) { return nyi(); }
}  // namespace qisg
