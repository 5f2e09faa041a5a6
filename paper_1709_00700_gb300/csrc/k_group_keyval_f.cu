// Grouped shape: SUM(val), COUNT(*) GROUP BY key with a range filter on val
// (selectivity knob of the random query suite).
#include "k_group.cuh"

namespace pv {

using ShKeyValF = Shape<Cols<TI64, TI32>, Where<P<0>>, Probes<>, Key<X<1>>, Aggs<Sum<Mul<X<0>>>, Count>, Proj<>>;

void register_group_keyval_f() { reg_grouped<ShKeyValF, 1>(); }

}  // namespace pv
