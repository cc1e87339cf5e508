// Group engine instantiations: Kuhn-Munkres (paper Sec. 2.3 / Sec. 4.1).
#define OT_ALGO ot::kAlgoKM
#define OT_LAUNCH_NAME launch_group_km
#include "ot_group_launch.inc"
