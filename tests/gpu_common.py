"""GPU-test helpers: the package's workload loader plus torch/numpy glue."""
from paper_2405_04463_gb300.workload import (db_bits_device, dev_u64, encode_gpu, galois, lib, load_workload,  # noqa: F401
                                             make_ctx, plain_mask_u16, query_shares_gpu, tags_for, torch_mod,
                                             u16)
