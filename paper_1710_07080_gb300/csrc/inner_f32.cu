// FP32 instantiation of the inner solve (mixed precision: FP32 inner, FP64 outer).
#include "inner_impl.cuh"
namespace isira {
ISIRA_INSTANTIATE_INNER(float)
}
