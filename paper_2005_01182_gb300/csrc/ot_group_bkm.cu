// Group engine instantiations: batched KM, exact mode (paper Sec. 2.3).
#define OT_ALGO ot::kAlgoBKM
#define OT_LAUNCH_NAME launch_group_bkm
#include "ot_group_launch.inc"
