// Grouped shape: SUM(val), COUNT(*) GROUP BY key over (key int32, val
// int64), the Aggregation Query 1/2 shape of Section 9.2.1 with the group
// count as a parameter.
#include "k_group.cuh"

namespace pv {

using ShKeyVal = Shape<Cols<TI32, TI64>, Where<>, Probes<>, Key<X<0>>, Aggs<Sum<Mul<X<1>>>, Count>, Proj<>>;

void register_group_keyval() { reg_grouped<ShKeyVal>(); }

}  // namespace pv
