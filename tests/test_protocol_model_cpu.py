"""Race checking of the tensor-core kernels' warp-role protocols on the CPU
(tests/_protocol_model.py: exact mbarrier parity semantics, TMA loads landing
in any order, MMAs completing in issue order, a data tag on every staging
slot, A chunk, accumulator and table).  The kernels' current protocols must
run clean under many random interleavings; the two earlier forms that the
model showed to be wrong must be caught."""
import pytest

import _protocol_model as P


@pytest.mark.parametrize("n", [8, 16, 32, 64])
@pytest.mark.parametrize("stages", [2, 4, 6, 8])
def test_single_lattice_step_is_race_free(n, stages):
    items = [(n, 0)] * 5 + [(n, 1)] * 3 + [(n, 0)] * 2          # class switches and back
    for seed in range(8):
        P.bf16_step(items, stages, seed)


@pytest.mark.parametrize("stages", [2, 4, 6, 8])
def test_batch_with_mixed_direction_counts_is_race_free(stages):
    items = ([(8, (0, 0))] * 4 + [(16, (1, 0))] * 3 + [(16, (1, 1))] * 2 + [(32, (2, 0))] * 3 +
             [(8, (3, 0))] * 2 + [(32, (4, 0))] * 2)
    for seed in range(12):
        P.bf16_step(items, stages, seed)


def test_shared_staging_ring_is_caught():
    """The earlier batch form in which both converter groups used one ring of
    staging slots: a group could pass a slot's parity test a full phase early
    when the other group lagged (seen on the GPU as faults)."""
    items = [(8, (0, 0))] * 4 + [(16, (1, 0))] * 3 + [(32, (2, 0))] * 3
    caught = 0
    for stages in (2, 3, 4):
        for seed in range(60):
            try:
                P.bf16_step(items, stages, seed, shared_ring=True)
            except P.ProtocolError:
                caught += 1
    assert caught > 0


@pytest.mark.parametrize("n", [8, 16, 32, 64])
@pytest.mark.parametrize("stages", [2, 4, 8])
def test_fp8_step_is_race_free(n, stages):
    items = [(n, 0)] * 4 + [(n, 1)] * 3
    for seed in range(8):
        P.fp8_step(items, stages, seed)


def test_fp8_without_the_t_ready_gate_is_caught():
    """The first FP8 form let a converter warp with no slot in a tile (group 1
    at n = 8) arrive on t_ready for later tiles at once, completing a tile's
    phase before the other group wrote the A operand; it showed only with
    several tiles per CTA."""
    with pytest.raises(P.ProtocolError):
        for seed in range(10):
            P.fp8_step([(8, 0)] * 4, 4, seed, gate_t_ready=False)
    for seed in range(10):                       # one tile per CTA hid it
        P.fp8_step([(8, 0)], 4, seed, gate_t_ready=False)


@pytest.mark.parametrize("stages", [2, 4])
def test_cta_pair_step_is_race_free(stages):
    """The headline CTA-pair kernel: forwarded readiness of the odd CTA
    (t_local -> t_ready, count 9), forwarded table half (z_full count 2),
    multicast commits to both CTAs' barriers."""
    for seed in range(10):
        P.pair_step([0, 0, 0, 1, 1, 0, 0], stages, seed)
    # orders where one role lags far behind the rest
    for slow in ("epi0", "epi1", "conv1", "forwarder", "producer1", "mma"):
        for seed in range(5):
            P.pair_step([0, 0, 1, 1, 0, 0], stages, seed, slow={slow: 0.01})


@pytest.mark.parametrize("n", [16, 32])
@pytest.mark.parametrize("stages", [4, 8])
def test_gather_form_is_race_free(n, stages):
    """The single-CTA step in the gather form of bilinear streaming:
    four-direction slots, two per converter group and chunk, and the ghost
    fill of edge tiles met on each group's fill barrier; also with one role
    lagging far behind."""
    items = [(n, 0), (n, 0), (n, 1), (n, 1), (n, 0)]
    for seed in range(8):
        P.bf16_step(items, stages, seed, gather=True, edge_tiles={0, 2, 3})
    for slow in ("conv01", "conv10", "epi", "mma", "producer"):
        for seed in range(3):
            P.bf16_step(items, stages, seed, gather=True, edge_tiles={1, 2}, slow={slow: 0.01})


def test_gather_model_sees_unfinished_fill():
    """Converter warps that read the window of an edge tile without waiting
    for the group's fill barrier: with one warp of the group lagging, the
    model must report a window part not yet filled."""
    with pytest.raises(P.ProtocolError, match="window part"):
        for seed in range(20):
            P.bf16_step([(32, 0)] * 3, 4, seed, gather=True, edge_tiles={0, 1, 2}, skip_fill_wait=True,
                        slow={"conv31": 0.01})


def test_gather_model_sees_wrong_ring():
    """A producer that hands the gather form's slots to the groups of the
    eight-direction form (j & 1) feeds a group slots of the other group's
    directions: the model must report it."""
    with pytest.raises(P.ProtocolError):
        P.bf16_step([(32, 0)] * 3, 4, 0, gather=True, gather_ring_flaw=True)


def test_cta_pair_model_sees_unreleased_accumulator():
    """Converters that write a tile's accumulator init before the epilogue
    of two tiles earlier has read that buffer: with the epilogue lagging, the
    model must report the overwrite."""
    with pytest.raises(P.ProtocolError, match="accumulator"):
        for seed in range(20):
            P.pair_step([0] * 6, 2, seed, gate_acc_empty=False, slow={"epi1": 0.01})


@pytest.mark.parametrize("n", [8, 16, 32, 64])
@pytest.mark.parametrize("stages", [2, 4])
def test_fp8x_step_is_race_free(n, stages):
    """The split-FP8 kernel: slots in hand-back order, staging released before
    the hand-off wait, packed scale cells per group, two-slot epilogue loads;
    also with one role lagging far behind."""
    for seed in range(6):
        P.fp8x_step([(n, 0), (n, 0), (n, 1), (n, 1), (n, 0)], stages, seed)
    for slow in ("epi", "conv1", "mma", "producer"):
        P.fp8x_step([(n, 0), (n, 0), (n, 1)], stages, 0, slow={slow: 0.01})


def test_fp8x_model_sees_early_handback():
    """An epilogue that hands a slot back before reading its columns lets the
    next tile's init overwrite them: the model must report it."""
    with pytest.raises(P.ProtocolError, match="accumulator"):
        for seed in range(5):
            P.fp8x_step([(64, 0)] * 4, 2, seed, early_handback=True)


@pytest.mark.parametrize("n", [8, 16, 32])
@pytest.mark.parametrize("stages", [2, 4, 6])
def test_tf32_step_is_race_free(n, stages):
    """The 3xTF32 kernel: ring of split chunks (a_full / a_empty), double D
    and E, chunk-wise MMAs from a zero accumulator; also with one role
    lagging far behind."""
    for seed in range(6):
        P.tf32_step([(n, 0), (n, 0), (n, 1), (n, 1), (n, 0)], stages, seed)
    for slow in ("epi", "conv1", "mma", "producer"):
        P.tf32_step([(n, 0), (n, 0), (n, 1)], stages, 0, slow={slow: 0.01})


def test_tf32_model_sees_ungated_ring():
    """At n = 32 (one ring slot per group) converters that skip the wait for
    the MMAs on their ring slot overwrite a chunk the MMA has not read: the
    model must report it.  (At n <= 16 the wait on the epilogue of tile
    i - 2 already implies it.)"""
    with pytest.raises(P.ProtocolError, match="ring slot"):
        for seed in range(5):
            P.tf32_step([(32, 0)] * 4, 2, seed, gate_ring=False)


@pytest.mark.parametrize("stages", [2, 4])
def test_table_gradient_is_race_free(stages):
    """The adjoint's tensor-core table gradient: staging ring, double-buffered
    operands, one pass per class present in a chunk (mixed chunks make two);
    also with one role lagging far behind."""
    masks = [1, 1, 3, 2, 2, 3, 1, 2, 1, 1]
    for seed in range(6):
        P.table_step(masks, stages, seed)
    for slow in ("conv3", "mma", "producer"):
        P.table_step(masks, stages, 0, slow={slow: 0.01})


def test_table_gradient_model_sees_ungated_buffer():
    """Converters that overwrite an operand buffer without waiting for the
    MMAs of the pass two before it: with the MMA thread lagging, the model
    must report the overwrite."""
    with pytest.raises(P.ProtocolError, match="operand buffer"):
        for seed in range(10):
            P.table_step([1] * 8, 4, seed, gate_done=False, slow={"mma": 0.01})
