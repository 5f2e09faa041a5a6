// Grouped shape of the TPC-H Q5-shaped multi-pipeline query (Section 9.2.1):
// line items probe the orders selected by the earlier pipelines and group on
// the nation the probe binds, SUM(extendedprice * (100 - discount)), COUNT(*).
#include "k_group.cuh"

namespace pv {

using ShQ5Lines = Shape<Cols<TI32, TI64, TI64>, Where<>, Probes<0>, Key<PL<0, 0>>,
                        Aggs<Sum<Mul<X<1>, CMX<2, 0>>>, Count>, Proj<>>;

void register_group_q5() { reg_grouped<ShQ5Lines, 1>(); }

}  // namespace pv
