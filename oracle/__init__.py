"""FP64 CPU oracle of the MLPF full-event transformer forward.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
this package; only the tests, the smoke check and the benchmark's CPU-baseline
leg do.  It shares no code with the CUDA library: it reads the same seeded
weights (float32 values widened to float64) and the same synthetic events.

Every function is the plain definition of one step of the method, written for
readability, in float64, with numpy matmul as the only library primitive
(scipy's erf for the exact GELU).  See forward.py for the per-step citations.
"""
from .forward import (  # noqa: F401
    layer_norm, gelu, relu, linear, softmax_rows, sdpa, attention_matrix,
    multi_head_attention, encoder_block, encoder_stack, embed, reg_embed,
    ffn_head, forward_event, decode, event_sums, forward, OracleOutput, is_track, embed_per_type,
    raw_from_decoded, log_softmax_rows, distill_loss, supervised_loss, softplus,
    SUP_BETA, SUP_FOCAL, SUP_DELTA, WINDOW_BLOCK, eta_order, window_mask,
)
