"""GB300-native multiplication of sparse Laurent polynomials and Poisson series.

Kronecker substitution followed by a schoolbook product accumulated in a
dense shared-memory array or an open-addressing hash table (Biscani, Sec. 2
and Sec. 3), implemented as hand-written CUDA for sm_103a behind the C ABI of
include/kron.h.  This package is the thin Python binding of that library.
"""
from .binding import (  # noqa: F401
    KR_OK, KR_ERR_INVALID, KR_ERR_RANGE, KR_ERR_OVERFLOW, KR_ERR_DUP, KR_ERR_OOM,
    KR_ERR_CAPACITY, KR_ERR_TIMEOUT, KR_ERR_CUDA, KR_ERR_TABLE_FULL, KR_ERR_TOO_LARGE,
    KR_PATH_AUTO, KR_PATH_DENSE, KR_PATH_HASH, KR_MAXV,
    Context, KronError, context, load, lib_path,
    kron_plan, kron_encode, kron_decode, poly_mul, poisson_mul, kr_probe_smem_atomic_rate,
    kr_probe_smem_accumulate_rate, kr_probe_table_update_rate, kr_probe_alu_rate,
    kr_selftest_bounded_wait,
    kron_dense_product_static, kron_mul_batch, PreparedBatch,
)
