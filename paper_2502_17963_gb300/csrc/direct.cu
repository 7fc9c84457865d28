// Direct (on-the-fly) DF mode: placeholder.
#include "bqc_internal.h"
#include "df_internal.h"

namespace bqc {
int direct_setup(Df *, cudaStream_t) { return BQC_E_UNSUPPORTED; }
int jk_direct(Df *, const double *, int, double *, double *, cudaStream_t) {
  return BQC_E_UNSUPPORTED;
}
}  // namespace bqc
