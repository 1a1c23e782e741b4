"""GPU-test helpers: the package's workload loader plus torch/numpy glue."""
from paper_2405_04463_gb300.workload import (db_bits_device, dev_u64, encode_gpu, encode_gpu32,  # noqa: F401
                                             galois, lib, lift_shares, load_workload, make_ctx, plain_mask_u16,
                                             query_shares_gpu, tags_for, torch_mod, u16)
