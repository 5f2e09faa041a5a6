// Grouped shape with a composite key of three fact columns:
// SUM(val), COUNT(*) GROUP BY a, b, c over (a, b, c int32, val int64).
// The key is the mixed-radix code of the three parts over their value spans.
#include "k_group.cuh"

namespace pv {

using ShKeys3 = Shape<Cols<TI32, TI32, TI32, TI64>, Where<>, Probes<>, Key<X<0>, X<1>, X<2>>,
                      Aggs<Sum<Mul<X<3>>>, Count>, Proj<>>;

void register_group_keys3() { reg_grouped<ShKeys3, 1>(); }

}  // namespace pv
