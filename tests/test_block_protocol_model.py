"""The intra-block protocol of the persistent kernels under random schedules (tests/block_protocol_model.py).

The PH lane kernel draws tickets three iterations ahead into a ring of eight slots, the batch kernel
two ahead into a ring of eight; the cyclic-reduction cascade kernel draws two ahead into a ring of
four.  All three correct
a tile one iteration after its fold (two row buffers) and keep two slots of local carries and of
incoming states, each slot with its own barrier.  The planted variants are mistakes of the kind
the model is there to catch: a single incoming-state barrier (the cyclic-reduction kernel had one,
never seen to misbehave on the GPU; its fix is checked here), a deeper pipeline without more
slots, and a ticket ring too small for its lookahead.
"""
import random

import pytest

from .block_protocol_model import Hazard, run_block

SEEDS = 300


def _cases(seed0):
    for seed in range(seed0, seed0 + SEEDS):
        r = random.Random(seed)
        yield r.choice([1, 2, 3, 7, 8]), r.randrange(0, 40), seed


def _hazards(**kw):
    found = []
    for W, n_tiles, seed in _cases(1000):
        try:
            run_block(W, n_tiles, seed=seed, **kw)
        except Hazard as e:
            found.append(str(e))
    return found


@pytest.mark.parametrize("name,kw", [
    ("PH lane kernel", dict(R=8, A=3, D=2, NS=2, NZ=2)),
    ("batch kernel", dict(R=8, A=2, D=2, NS=2, NZ=2)),
    ("cyclic-reduction cascade kernel", dict(R=4, A=2, D=2, NS=2, NZ=2)),
])
def test_kernel_protocols_are_hazard_free(name, kw):
    assert _hazards(**kw) == [], name


@pytest.mark.parametrize("what,kw,hint", [
    ("one incoming-state barrier", dict(R=8, A=3, D=2, NS=2, NZ=1), "waits for phase"),
    ("a three-stage pipeline on two slots", dict(R=8, A=3, D=3, NS=2, NZ=2), "not yet consumed"),
    ("a ring of four with tickets three ahead", dict(R=4, A=3, D=2, NS=2, NZ=2), "ticket slot"),
])
def test_planted_protocol_mistakes_are_caught(what, kw, hint):
    found = _hazards(**kw)
    assert found, what
    assert any(hint in f for f in found), (what, found[:3])


def test_a_deeper_pipeline_with_four_slots_is_hazard_free():
    # the three-stage pipeline (correction two iterations after the fold) with slots mod 4
    assert _hazards(R=8, A=3, D=3, NS=4, NZ=4) == []


def test_loading_into_the_buffer_the_correction_freed_is_hazard_free():
    # the next tile's samples go straight into the row buffer the correction has just read
    assert _hazards(R=8, A=3, D=2, NS=2, NZ=2, load="after_correction") == []
    # issued before that correction, the load would overwrite a tile still to be corrected
    found = _hazards(R=8, A=3, D=2, NS=2, NZ=2, load="early")
    assert found and any("still holds" in f for f in found)


def test_every_tile_is_corrected_once_for_empty_and_single_tile_launches():
    for n_tiles in (0, 1, 2):
        for W in (1, 7):
            run_block(W, n_tiles, seed=n_tiles * 10 + W)
