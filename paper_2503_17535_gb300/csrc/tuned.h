// Shape choices of the batched LU and the tensor-core routing thresholds on
// GB300 (hps_tune_set in include/hps.h).  Written by
// paper_2503_17535_gb300/autotune.py from timed builds of the benchmark
// workloads (summed median build time, ms, at the chosen values:
// {"helmholtz2d_iti_p16_depth6": 211.52, "elliptic3d_dtn_p8_depth3": 168.99, "adaptive3d_dtn_p8": 135.35}); rerun it to regenerate.
#pragma once

#define HPS_TUNED_LU_CLUSTER_PANEL 1
#define HPS_TUNED_LU_BASE_PANELS_FEW 32
#define HPS_TUNED_LU_FEW_MIN_N 4096
#define HPS_TUNED_LU_BASE_PANELS_MANY 8
#define HPS_TUNED_TC_MIN_WORK_REAL 100
#define HPS_TUNED_TC_MIN_WORK_CPLX 25
#define HPS_TUNED_TC_MIN_K 16
