// Temporally blocked filter kernels for bf16 storage (see pm_tb.cuh).
#define AFD_TB_STORE STORE_BF16
#define AFD_TB_FN(name) tb_##name##_bf16
#include "pm_tb_impl.cuh"
