"""GB300-native exact three-hop top-K path search (libmhr.so, sm_103a).

The compute path is the CUDA library behind the C ABI in include/mhr.h; this
package only marshals arguments to it (see _mhr.py) and compiles it
(build.py).  Importing the package loads the library and fails loudly when it
cannot be built or loaded: there is no CPU fallback.
"""

from ._mhr import (  # noqa: F401
    EXPORTS,
    Graph,
    MhrError,
    PATH_DTYPE,
    TAIL_DTYPE,
    MHR_K_MAX,
    MHR_TAIL_K_MAX,
    MHR_OK,
    MHR_EINVAL,
    MHR_ENOMEM,
    MHR_ECUDA,
    MHR_ETIMEOUT,
    MHR_ERANGE,
    MHR_SCORE_TRANSE_L1,
    MHR_SCORE_DISTMULT,
    QueryOpts,
    Stats,
    lib_path,
    load_kg,
    load_library,
    mhr_edge_scores,
    mhr_graph_free,
    mhr_graph_get_info,
    mhr_graph_load,
    mhr_last_error,
    mhr_topk_paths,
    mhr_topk_paths_batched,
    mhr_topk_paths_noalloc,
    mhr_autotune,
    mhr_training_labels,
    mhr_mlp_features,
    mhr_mlp_forward,
    mhr_mlp_backward,
    mhr_mlp_adam,
    mhr_mlp_to_bf16,
    MLP,
    mhr_version,
    paths_from_device,
    mhr_tail_topk,
    tails_from_device,
    mhr_beam_paths,
    mhr_merge_paths,
    beams_from_device,
    BEAM_DTYPE,
)

from .learn import OrderingMLP, train_ordering_mlp  # noqa: E402,F401
from .partition import topk_paths_partitioned  # noqa: E402,F401

load_library()
