"""GPU (sm_103a) overlap-add room-simulator filter-and-mix.

Public API (loaded lazily so that importing the package, or its synthetic
input generators, does not need a GPU):
  Plan                 -- a plan for a batch shape (wraps rsim_plan)
  filter_mix           -- forward with allocated outputs
  RsimFilterMix        -- torch.autograd.Function with the hand-written adjoint
  filter_mix_autograd  -- RsimFilterMix.apply
  image_rirs           -- image-method RIRs (wraps rsim_image_rirs)
Plan also carries the log-Mel front end (Plan.log_mel, Plan.log_mel_rows) and
the gain modes: 0 gains from SNRs on the dry signals, 1 given per source,
2 given per (source, microphone), 3 from SNRs on the reverberant signal at
microphone snr_ref_mic.
"""
_API = ("Plan", "filter_mix", "RsimFilterMix", "filter_mix_autograd", "image_rirs")

__all__ = list(_API) + ["synth", "build"]


def __getattr__(name):
    if name in _API:
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
