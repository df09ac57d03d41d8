"""Seeded synthetic inputs for the transient F-statistic map.

This package makes the per-SFT "atoms" (Sec. 3: three real rows a^2, b^2, ab
and the complex Fa, Fb, i.e. 7 reals per SFT) that both the CPU oracle and the
CUDA library consume.  It models data, not the F-map: timestamps with gaps,
the daily antenna-pattern modulation of each detector, Gaussian noise, and an
optional transient signal whose amplitude follows the paper's window shapes
(Eq. winrect / winexp).  No windowed sum, determinant or F-statistic is
computed here.

Everything is drawn from numpy's counter-based Philox generator keyed by
(base seed, stream index), so one template or one instance can be regenerated
alone and a sample of a workload is bit-identical to the same part of the full
workload.
"""

from .atoms import (  # noqa: F401
    T_SFT,
    OMEGA_SID,
    RECT,
    EXP,
    TABLE,
    BASE_SEED,
    Grid,
    Injection,
    Instance,
    rect,
    exp_,
    envelope,
    make_instance,
    uneven_spec,
    instance_from_spec,
    config_small_rect,
    config_exp16,
    config_batched,
    config_uneven,
    config_serving_stream,
    philox,
)
