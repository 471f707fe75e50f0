"""The autograd wrappers rebuild the operator exactly when the potential's values differ from those of
the last build: a new tensor (even one that reuses freed memory), or an in-place change. CPU only:
a stand-in context records the builds."""
import torch

from paper_2010_09701_gb300.autograd import _ensure_built
from paper_2010_09701_gb300.binding import Context


class RecordingContext:
    built_from = Context.built_from

    def __init__(self):
        self._built_v, self._built_version, self.built_store = None, -1, 5
        self.builds = []

    def build_hamiltonian(self, veff, store):
        self.builds.append(store)
        self._built_v, self._built_version, self.built_store = veff, veff._version, store


def test_rebuild_only_for_new_values():
    ctx = RecordingContext()
    V = torch.zeros(1000, dtype=torch.float64)
    _ensure_built(ctx, V)
    _ensure_built(ctx, V)
    assert ctx.builds == [5]                    # same values: one build, with the last storage
    V.add_(1.0)
    _ensure_built(ctx, V)
    assert len(ctx.builds) == 2                 # in-place change
    for s in (1.0, -1.0):                       # temporaries made one after the other
        Vs = V + s
        _ensure_built(ctx, Vs)
        del Vs
    assert len(ctx.builds) == 4
    _ensure_built(ctx, V.detach())
    assert len(ctx.builds) == 5
    _ensure_built(ctx, V)                       # an alias of the built tensor: same values
    assert len(ctx.builds) == 5
