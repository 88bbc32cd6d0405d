// Split-precision engines (FP16x3 / BF16x3 tensor-core products).
#include "precision.h"

namespace xl {

Engine* make_split_engine(int) { return nullptr; }
cudaError_t alloc_matset_split(MatSet&) { return cudaErrorNotSupported; }
void free_matset_split(MatSet&) {}

}  // namespace xl
