"""GB300 (sm_103a) histogram-sampling muon transport.

The compute path is the C-ABI library libmt.so (include/mt.h, sources in csrc/);
this package is its thin Python binding.  Import does not touch the GPU; the
first call that needs the library loads it and raises if it was not built.
"""
from ._binding import (  # noqa: F401
    MT_ALIVE, MT_STOPPED, MT_EXIT_Z, MT_EXIT_XY, MT_MAX_STEPS, MT_INVALID,
    MtError, declared_symbols, library_path, load_library,
    mt_abi_version, mt_last_error, mt_create, mt_destroy, mt_device_bytes,
    mt_transport, mt_transport_scaled, mt_transport_cfg, mt_transport_workspace_bytes, mt_transport_launches,
    MT_LAUNCH_AUTO, MT_LAUNCH_STATIC, MT_LAUNCH_PERSISTENT, MT_LAUNCH_COMPACT, MT_SAMPLER_ICDF, MT_SAMPLER_ALIAS,
    MT_ORDER_AUTO, MT_ORDER_ALWAYS, MT_ORDER_NEVER,
    mt_transport_noalloc, MT_NOALLOC_MAX_MUONS,
    mt_ckpt_bytes, mt_transport_ckpt, mt_adjoint_ckpt, mt_transport_adjoint, mt_acceptance_loss,
    mt_tape_bytes, mt_transport_tape, mt_adjoint_tape,
    mt_build_histograms, mt_pilot_phi, mt_bv_edges,
    mt_batch_create, mt_batch_set_instance, mt_batch_destroy, mt_batch_device_bytes, mt_batch_workspace_bytes,
    mt_transport_batched, mt_batch_autotune, MT_BATCH_STAGE_SHARED, MT_BATCH_STAGE_GLOBAL,
)
from .api import (World, Batch, muons_to_device, muons_to_host, empty_like_soa,  # noqa: F401
                  build_histogram_set, bounded_variation_edges)
from .autograd import MuonTransportFn, AcceptanceLossFn, transport_differentiable, acceptance_loss  # noqa: F401,E402
