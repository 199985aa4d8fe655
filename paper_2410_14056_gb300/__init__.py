"""GB300-native random-walk spanning centrality (arXiv 2410.14056 hot path).

The compute path is the CUDA library ``libbouquet.so`` (C ABI in
``include/bouquet.h``); ``bouquet`` is its thin ctypes binding.  Build the
library with ``paper_2410_14056_gb300.build.build()``.
"""

from .bouquet import (  # noqa: F401
    AESC_NAIVE, BORROW, DEVICE_PTRS, EBUSY, ECUDA, EGRAPH, EINVAL, ENOEDGE, ENOMEM, EOVERFLOW, ETIMEOUT, HOST_IO,
    HOST_PTRS, MODE_BOUQUET, MODE_NAIVE, OK, PLAN_CERTIFIED, PLAN_SCHEDULED, PUSH_SUPPORT_CAP, REQUIRE_CONNECTED,
    SAMPLER_COUPLED, SAMPLER_IND, SAMPLER_SABA, SKIP_VALIDATE, VISIT_START, WALK_KERNELS, Batch, BouquetError, Graph,
    Sampler, Schedule, Server, ServerConfig, aesc_estimate, aesc_estimate_host, aesc_estimate_push,
    aesc_estimate_push_host, aesc_estimate_shared, aesc_estimate_shared_host, aesc_plan, aesc_plan_pilot,
    autotune_aesc, autotune_walks, get_tuning, load_library, profile_enable, profile_read, read_bandwidth,
    set_tuning, sync, version, walk_batch, walk_batch_host, walk_batch_noalloc,
)
