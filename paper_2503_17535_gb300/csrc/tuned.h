// Shape choices of the batched LU and the tensor-core routing thresholds on
// GB300 (hps_tune_set in include/hps.h).  Written by
// paper_2503_17535_gb300/autotune.py from timed builds of the benchmark
// workloads (summed median build time, ms, at the chosen values:
// {"helmholtz2d_iti_p16_depth6": 171.74, "elliptic3d_dtn_p8_depth3": 150.87, "adaptive3d_dtn_p8": 122.98}); rerun it to regenerate.
#pragma once

#define HPS_TUNED_LU_CLUSTER_PANEL 1
#define HPS_TUNED_LU_BASE_PANELS_FEW 32
#define HPS_TUNED_LU_FEW_MIN_N 4096
#define HPS_TUNED_LU_BASE_PANELS_MANY 8
#define HPS_TUNED_TC_MIN_WORK_REAL 50
#define HPS_TUNED_TC_MIN_WORK_CPLX 50
#define HPS_TUNED_TC_MIN_K 16
#define HPS_TUNED_TC_CHUNK_MB 1024
#define HPS_TUNED_TC_PERSIST_MIN_K 0
#define HPS_TUNED_LU_PANEL_NB_FEW 32
