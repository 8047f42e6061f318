"""GB300-native symmetric block-sparse tensors: U(1), SU(2), fermion parity
and SU(2) x U(1).

Hot path of S. Singh's tensor-network symmetry method (arXiv:1203.2222):
integer sector tables, block gathers with SU(2) recoupling, a grouped
per-sector GEMM on tcgen05 tensor cores, the scatter back, and the adjoint;
also the blockwise SVD and symmetric eigendecomposition with truncation.
The compute lives in ``_build/libsymtensor.so`` (C ABI: include/symtensor.h);
this package is its Python front end.
"""
from .symtensor import (BF16X3, FP64, KERNEL_SYMBOLS, KERNELS, PHASES, SU2, U1, BatchPlan,  # noqa: F401
                        Plan, Structure, SymError, SymTensor, cached_plans, contract, contract_batch,
                        contract_batch_plan, contract_plan, device_status, fuse, fuse_plan, permute,
                        permute_plan, split, split_plan, su2_F, su2_gamma, svd, svd_plan, SVDPlan, eig,
                        eig_plan, EigPlan, tune_epoch, tune_get, tune_set, Z2F, SU2U1, su2u1_label)
