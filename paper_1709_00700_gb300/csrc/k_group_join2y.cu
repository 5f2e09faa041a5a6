// Grouped join shape of Table 2's pipeline program grouping on the payload
// of the second build, with SUM, COUNT, MIN and MAX: filter, two probes.
#include "k_group.cuh"

namespace pv {

using ShTable2Y = Shape<Cols<TI32, TI32, TI32, TI64>, Where<P<0>>, Probes<1, 2>, Key<PL<1, 0>>,
                        Aggs<Sum<Mul<X<3>>>, Count, Min<Mul<X<3>>>, Max<Mul<X<3>>>>, Proj<>>;

void register_group_join2y() { reg_grouped<ShTable2Y, 1>(); }

}  // namespace pv
