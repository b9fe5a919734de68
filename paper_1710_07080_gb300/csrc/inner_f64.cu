// FP64 instantiation of the inner solve (plain FP64 mode).
#include "inner_impl.cuh"
namespace isira {
ISIRA_INSTANTIATE_INNER(double)
}
