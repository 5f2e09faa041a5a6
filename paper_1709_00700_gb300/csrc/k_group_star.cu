// Grouped join shape: the four-probe star join (SSB Q4.1 shape, Section
// 9.2.1) probing four build-side tables and grouping on two payloads.
#include "k_group.cuh"

namespace pv {

using ShStar4 = Shape<Cols<TI32, TI32, TI32, TI32, TI64>, Where<>, Probes<0, 1, 2, 3>, Key<PL<2, 0>, PL<3, 0>>,
                      Aggs<Sum<Mul<X<4>>>, Count>, Proj<>>;

void register_group_star() { reg_grouped<ShStar4, 1>(); }

}  // namespace pv
