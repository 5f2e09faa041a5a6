// Grouped join shape of Table 2's pipeline program grouping on the payload
// of the first build: filter, two probes.
#include "k_group.cuh"

namespace pv {

using ShTable2X = Shape<Cols<TI32, TI32, TI32, TI64>, Where<P<0>>, Probes<1, 2>, Key<PL<0, 0>>,
                        Aggs<Sum<Mul<X<3>>>, Count>, Proj<>>;

void register_group_join2() { reg_grouped<ShTable2X, 1>(); }

}  // namespace pv
