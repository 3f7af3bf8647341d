"""Model checker: every algorithm passes on all interleavings of tiny inputs, and every
planted mistake (in the oracle's models, on the CPU) is caught."""
import pytest

from oracle import model_check as mc

W = 2 ** 32 - 3  # counters start just below 2^32 so that they wrap during the run

CORRECT = [
    ("spin_exch", mc.SpinMutex(), 3, 2),
    ("spin_exch_atomic_unlock", mc.SpinMutex(atomic_unlock=True), 3, 2),
    ("spin_backoff", mc.SpinMutex(backoff=True), 3, 2),
    ("spin_cas", mc.SpinMutex(cas=True), 3, 2),
    ("ticket", mc.TicketMutex(), 3, 2),
    ("ticket_literal_unlock", mc.TicketMutex(literal=True), 3, 2),
    ("ticket_wrap", mc.TicketMutex(base=W), 3, 2),
    ("ticket_carry", mc.CarryTicketMutex(), 3, 2),
    ("ticket_carry_wrap", mc.CarryTicketMutex(base=W), 3, 2),
    ("queue", mc.QueueMutex(q=4), 3, 2),
    ("queue_wrap", mc.QueueMutex(q=4, base=W), 3, 2),
    ("queue_exact_fit", mc.QueueMutex(q=2, base=W), 2, 3),
    ("ring", mc.RingMutex(q=4), 3, 2),
    ("condvar_1p1c", mc.CondVarQueue(P=1, C=1), 2, 3),
    ("condvar_1p1c_cap2", mc.CondVarQueue(P=1, C=2), 2, 3),
    ("condvar_2p2c", mc.CondVarQueue(P=2, C=1), 4, 2),
    ("condvar_2p2c_broadcast", mc.CondVarQueue(P=2, C=1, broadcast=True), 4, 2),
    ("cohort_budget_1", mc.CohortMutex(budget=1), 4, 1),
    ("cohort_budget_2", mc.CohortMutex(budget=2), 3, 2),
    ("cohort_budget_2_4x2", mc.CohortMutex(budget=2), 4, 2),
    ("cohort_budget_3", mc.CohortMutex(budget=3), 3, 2),
    ("cohort_wrap", mc.CohortMutex(budget=2, base=W, gbase=0xFFFE), 3, 2),
    ("cohort_three_groups", mc.CohortMutex(budget=2, groups=3), 4, 2),
    ("mcs_cohort_one_cluster", mc.McsCohortMutex(cluster_of=(0, 0, 0)), 3, 2),
    ("mcs_cohort_two_clusters", mc.McsCohortMutex(cluster_of=(0, 0, 1)), 3, 2),
    ("mcs_cohort_three_clusters", mc.McsCohortMutex(cluster_of=(0, 1, 2)), 3, 2),
    ("mcs_cohort_four_blocks", mc.McsCohortMutex(cluster_of=(0, 0, 1, 1)), 4, 1),
    ("mcs_cohort_budget_1", mc.McsCohortMutex(budget=1), 3, 2),
    ("mcs_cohort_budget_3", mc.McsCohortMutex(cluster_of=(0, 0, 0), budget=3), 3, 2),
    ("mcs_cohort_three_rounds", mc.McsCohortMutex(cluster_of=(0, 0)), 2, 3),
    ("cohort_carry_budget_2", mc.CarryCohortMutex(budget=2), 3, 2),
    ("cohort_carry_budget_1", mc.CarryCohortMutex(budget=1), 4, 1),
    ("cohort_carry_budget_3", mc.CarryCohortMutex(budget=3), 3, 2),
    ("cohort_carry_three_groups", mc.CarryCohortMutex(budget=2, groups=3), 4, 1),
    ("hier_carry_one_die", mc.CarryMcsHierMutex(cluster_of=(0, 0, 1), die_of=(0, 0)), 3, 2),
    ("hier_carry_one_cluster", mc.CarryMcsHierMutex(cluster_of=(0, 0, 0), die_of=(0,)), 3, 2),
    ("hier_carry_two_dies", mc.CarryMcsHierMutex(cluster_of=(0, 0, 1), die_of=(0, 1)), 3, 2),
    ("hier_carry_three_clusters", mc.CarryMcsHierMutex(cluster_of=(0, 1, 2), die_of=(0, 0, 1)), 3, 2),
    ("hier_carry_four_blocks", mc.CarryMcsHierMutex(cluster_of=(0, 0, 1, 1), die_of=(0, 1)), 4, 1),
    ("hier_carry_budget_1", mc.CarryMcsHierMutex(cbudget=1, dbudget=1), 3, 2),
    ("hier_carry_cluster_budget_3", mc.CarryMcsHierMutex(cluster_of=(0, 0, 0), die_of=(0,), cbudget=3), 3, 2),
    ("hier_carry_three_rounds", mc.CarryMcsHierMutex(cluster_of=(0, 0), die_of=(0,)), 2, 3),
    ("spin_sem_1", mc.SpinSem(n=1), 3, 2),
    ("spin_sem_2", mc.SpinSem(n=2), 3, 2),
    ("spin_sem_2_backoff", mc.SpinSem(n=2, backoff=True), 3, 2),
    ("sleep_sem_1", mc.SleepSem(n=1), 3, 2),
    ("sleep_sem_2", mc.SleepSem(n=2), 3, 2),
    ("sleep_sem_wrap", mc.SleepSem(n=1, base=W), 3, 2),
    ("window_sem_1", mc.WindowSem(n=1), 3, 2),
    ("window_sem_2", mc.WindowSem(n=2), 3, 2),
    ("window_sem_2_of_4", mc.WindowSem(n=2), 4, 2),
    ("window_sem_wrap", mc.WindowSem(n=2, base=W), 3, 3),
    ("atomic_barrier", mc.AtomicBarrier(), 3, 2),
    ("atomic_barrier_wrap", mc.AtomicBarrier(base=2 ** 32 - 1), 3, 3),
    ("atomic_barrier_parity", mc.AtomicBarrier(parity=True), 4, 3),
    ("atomic_barrier_parity_wrap", mc.AtomicBarrier(parity=True, base=2 ** 32 - 2), 3, 4),
    ("flag_barrier", mc.FlagBarrier(), 3, 2),
    ("flag_barrier_broadcast", mc.FlagBarrier(broadcast=True), 3, 2),
    ("flag_barrier_wrap", mc.FlagBarrier(base=2 ** 32 - 1), 3, 3),
    ("tree_barrier_3", mc.TreeBarrier(fan=2), 3, 2),
    ("tree_barrier_4", mc.TreeBarrier(fan=2), 4, 2),
    ("tree_count_barrier_3", mc.TreeCountBarrier(fan=2), 3, 2),
    ("tree_count_barrier_4", mc.TreeCountBarrier(fan=2), 4, 2),
    ("tree_count_barrier_5", mc.TreeCountBarrier(fan=2), 5, 1),
    ("tree_count_barrier_fan3", mc.TreeCountBarrier(fan=3), 4, 2),
    ("tree_count_barrier_base", mc.TreeCountBarrier(fan=2, base=3), 4, 3),
    ("tree_count_barrier_one_node", mc.TreeCountBarrier(fan=4), 3, 3),
    ("cluster_barrier", mc.ClusterBarrier(c=2), 4, 2),
    ("cluster_count_barrier_poll", mc.ClusterCountBarrier(c=2), 4, 2),
    ("cluster_count_barrier_poll_base", mc.ClusterCountBarrier(c=2, base=3), 4, 3),
    ("cluster_count_barrier_three_clusters", mc.ClusterCountBarrier(c=2), 6, 1),
    ("cluster_count_barrier_c3", mc.ClusterCountBarrier(c=3), 6, 1),
    ("cluster_count_barrier_c1", mc.ClusterCountBarrier(c=1), 3, 2),
    ("cluster_count_barrier_second", mc.ClusterCountBarrier(c=2, release="cluster"), 4, 2),
    ("cluster_count_barrier_second_base", mc.ClusterCountBarrier(c=2, base=2, release="cluster"), 4, 3),
    ("sharded_barrier_2", mc.ShardedBarrier(shards=2), 3, 3),
    ("sharded_barrier_3", mc.ShardedBarrier(shards=3), 4, 2),
    ("sharded_barrier_1", mc.ShardedBarrier(shards=1), 3, 2),
    ("sharded_barrier_wrap", mc.ShardedBarrier(shards=2, base=2 ** 32 - 1), 3, 3),
    ("count_barrier", mc.CountBarrier(), 4, 3),
    ("exchange_in_order", mc.ExchangeBarrier(), 3, 3),
    ("exchange_counts_in_first", mc.ExchangeBarrier(late=(True, True, True)), 3, 3),
    ("exchange_mixed_orders", mc.ExchangeBarrier(late=(True, False, True)), 3, 3),
    ("exchange_base", mc.ExchangeBarrier(base=5, late=(False, True)), 2, 4),
    ("count_barrier_base", mc.CountBarrier(base=5), 3, 4),
    ("count_barrier_two_level", mc.CountBarrier(S=2), 4, 3),
    ("count_barrier_two_level_3", mc.CountBarrier(S=3, base=2), 4, 3),
    ("count_barrier_more_subs_than_blocks", mc.CountBarrier(S=4), 3, 3),
    ("split_barrier_1x1", mc.SplitBarrier(S=1, R=1), 4, 3),
    ("split_barrier_1x2", mc.SplitBarrier(S=1, R=2), 4, 3),
    ("split_barrier_2x2", mc.SplitBarrier(S=2, R=2), 4, 3),
    ("split_barrier_3x2", mc.SplitBarrier(S=3, R=2), 4, 3),
    ("split_barrier_wrap", mc.SplitBarrier(S=2, R=3, base=2 ** 32 - 2), 3, 4),
    ("die_barrier_alternating", mc.DieBarrier(), 4, 3),
    ("die_barrier_uneven", mc.DieBarrier(layout=(0, 0, 1)), 3, 4),
    ("die_barrier_one_die", mc.DieBarrier(layout=(1, 1, 1)), 3, 3),
    ("die_barrier_wrap", mc.DieBarrier(base=2 ** 32 - 2), 3, 4),
    # the serving ring's entry: both write orders of its two halves, both read orders
    ("ring_publish_lo_first", mc.RingPublish(), 2, 3),
    ("ring_publish_hi_first", mc.RingPublish(hi_first=True), 2, 3),
    ("ring_publish_read_hi_first", mc.RingPublish(read_hi_first=True), 2, 3),
    ("ring_publish_both_hi_first", mc.RingPublish(hi_first=True, read_hi_first=True), 2, 4),
    # a serving slot reused by requests of 1 and 2 chunks, two and three workers
    ("serve_slot_1_2", mc.ServeSlot(nch=(1, 2)), 3, 1),
    ("serve_slot_2_1", mc.ServeSlot(nch=(2, 1)), 3, 1),
    ("serve_slot_1_2_1", mc.ServeSlot(nch=(1, 2, 1)), 3, 1),
    ("serve_slot_three_workers", mc.ServeSlot(nch=(1, 2)), 4, 1),
]


@pytest.mark.parametrize("name,model,nproc,ops", CORRECT, ids=[c[0] for c in CORRECT])
def test_algorithm_is_safe_and_live(name, model, nproc, ops):
    r = mc.check(model, nproc, ops)
    assert r.ok, (r.violation, r.trace[-3:] if r.trace else r.stuck_state)
    assert r.states > 10


BROKEN = [
    ("test_then_set", mc.SpinMutex(broken="test_then_set"), 2, 1, "critical section"),
    ("ticket_no_advance", mc.TicketMutex(broken="no_advance"), 2, 2, "final state"),
    ("ticket_carry_split_read", mc.CarryTicketMutex(broken="split_read"), 2, 2, "entered with"),
    ("ticket_carry_turn_only", mc.CarryTicketMutex(broken="turn_only"), 2, 2, "entered with"),
    ("ring_no_clear", mc.RingMutex(q=2, broken="no_clear"), 2, 3, "grant"),
    ("condvar_release_before_ticket", mc.CondVarQueue(P=1, C=1, broken="signal_before_ticket"), 2, 3, "deadlock"),
    ("condvar_no_recheck", mc.CondVarQueue(P=2, C=1, broken="no_recheck"), 4, 2, "buffer count"),
    ("cohort_no_global", mc.CohortMutex(broken="no_global"), 2, 1, "critical section"),
    ("cohort_owned_on_release", mc.CohortMutex(broken="owned_on_release"), 2, 2, "critical section"),
    ("cohort_pass_always", mc.CohortMutex(broken="pass_always"), 2, 2, "final state"),
    ("cohort_skip_ticket", mc.CohortMutex(broken="skip_ticket"), 3, 2, "local ticket"),
    # The same mistakes with three groups, the shape of the cluster cohort lock.
    ("cohort3_no_global", mc.CohortMutex(broken="no_global", groups=3), 3, 1, "critical section"),
    ("cohort3_owned_on_release", mc.CohortMutex(broken="owned_on_release", groups=3), 3, 2, "critical section"),
    ("cohort3_pass_always", mc.CohortMutex(broken="pass_always", groups=3), 3, 2, "final state"),
    ("cohort3_skip_ticket", mc.CohortMutex(broken="skip_ticket", groups=3), 4, 2, "local ticket"),
    # Carrying cohort lock: a holder granted by the global lock that takes the local record's
    # sum, and a local pass that does not add the holder's own contribution.
    ("cohort_carry_global_reads_local", mc.CarryCohortMutex(broken="global_reads_local"), 3, 2, "entered with"),
    ("cohort_carry_pass_without_add", mc.CarryCohortMutex(broken="pass_without_add"), 3, 2, "entered with"),
    # MCS cluster cohort lock: the same three mistakes, and an owned record pushed after the
    # holder released the global lock.
    ("mcs_cohort_no_seq_check", mc.McsCohortMutex(broken="no_seq_check"), 3, 2, "critical section"),
    ("mcs_cohort_stale_link", mc.McsCohortMutex(broken="stale_link"), 3, 2, "cannot reach completion"),
    ("mcs_cohort_no_cas", mc.McsCohortMutex(cluster_of=(0, 0, 0), broken="no_cas"), 3, 2, "cannot reach completion"),
    ("mcs_cohort_owned_after_release", mc.McsCohortMutex(broken="owned_after_release"), 3, 2, "critical section"),
    # Three-level carrying lock: a waiter that takes any record in its node as its grant, a
    # holder that trusts a link left by an earlier round, and a holder without a linked
    # successor that leaves the tail naming itself.
    ("hier_carry_no_seq_check", mc.CarryMcsHierMutex(broken="no_seq_check"), 3, 2, "entered with"),
    ("hier_carry_stale_link", mc.CarryMcsHierMutex(broken="stale_link"), 3, 2, "cannot reach completion"),
    ("hier_carry_no_cas", mc.CarryMcsHierMutex(cluster_of=(0, 0, 0), die_of=(0,), broken="no_cas"), 3, 2,
     "cannot reach completion"),
    # Exchange barrier: one record per block instead of two by parity (a fast block overwrites
    # one still to be read), a reader that skips the epoch check (it can take last round's
    # value while the new record is in flight), a target one short.
    ("exchange_single_buffer", mc.ExchangeBarrier(broken="single_buffer"), 3, 3, "cannot reach completion"),
    ("exchange_no_epoch_check", mc.ExchangeBarrier(late=(True, False, True), broken="no_epoch_check"), 3, 3, "read"),
    ("exchange_off_by_one", mc.ExchangeBarrier(broken="off_by_one"), 3, 3, "passed round"),
    # Serving ring: an admitter that checks one sequence number (the other half may still be
    # the previous lap's), and a producer that reuses the slot before its request was taken.
    ("ring_publish_one_check", mc.RingPublish(broken="one_check"), 2, 3, "taken with"),
    ("ring_publish_one_check_read_hi", mc.RingPublish(read_hi_first=True, broken="one_check"), 2, 3, "taken with"),
    ("ring_publish_no_reuse_wait", mc.RingPublish(broken="no_reuse_wait"), 2, 3, "cannot reach completion"),
    # Serving slot: a worker that ignores its claim's generation (an over-claim of the last
    # request becomes a second claim of a chunk of the next), and an admitter that does not
    # reset the done count (the next request completes with a chunk missing).
    ("serve_slot_no_gen_check", mc.ServeSlot(nch=(1, 2), broken="no_gen_check"), 3, 1, "processed twice"),
    ("serve_slot_no_done_reset", mc.ServeSlot(nch=(1, 2), broken="no_done_reset"), 3, 1, "completed with"),
    ("sleep_sem_turn_ge", mc.SleepSem(n=1, broken="turn_ge"), 3, 1, "critical section"),
    ("window_sem_ge", mc.WindowSem(n=2, broken="window_ge"), 3, 1, "critical section"),
    ("barrier_no_wait", mc.AtomicBarrier(broken="no_wait"), 3, 1, "passed round"),
    ("barrier_late_reset_one_counter", mc.AtomicBarrier(broken="reset_one_counter"), 2, 3, "deadlock"),
    ("flag_skip_last", mc.FlagBarrier(broken="skip_last"), 3, 1, "passed round"),
    ("sharded_early", mc.ShardedBarrier(shards=2, broken="early"), 3, 1, "passed round"),
    ("die_no_top", mc.DieBarrier(broken="no_top"), 2, 2, "passed round"),
    ("split_no_top", mc.SplitBarrier(S=2, R=2, broken="no_top"), 3, 1, "passed round"),
    ("count_off_by_one", mc.CountBarrier(broken="off_by_one"), 3, 1, "passed round"),
    ("count_top_early", mc.CountBarrier(S=2, broken="top_early"), 4, 2, "passed round"),
    ("split_one_copy_early", mc.SplitBarrier(S=2, R=2, broken="one_copy_early"), 3, 3, "completion"),
    ("die_no_reset", mc.DieBarrier(broken="no_reset"), 2, 4, "final state"),
    ("sharded_counts_master", mc.ShardedBarrier(shards=2, broken="counts_master"), 3, 1, "final state"),
    # Queue lock: an unsigned poll lets a small ticket after the wrap through at once; an unlock
    # into the holder's own slot, or a successor slot that does not wrap to 0, wakes nobody.
    ("queue_unsigned_poll", mc.QueueMutex(q=4, base=W, broken="unsigned_ge"), 3, 2, "critical section"),
    ("queue_own_slot", mc.QueueMutex(q=4, broken="own_slot"), 2, 2, "final state"),
    ("queue_no_ring_wrap", mc.QueueMutex(q=2, broken="no_ring_wrap"), 2, 2, "final state"),
    # Spin-lock semaphore: a wait that keeps the permit, a post that does not return it, and a
    # wait at capacity that leaves the internal lock taken.
    ("spin_sem_keep_v", mc.SpinSem(n=1, broken="keep_v"), 2, 1, "critical section"),
    ("spin_sem_keep_v_n2", mc.SpinSem(n=2, broken="keep_v"), 3, 1, "critical section"),
    ("spin_sem_post_no_inc", mc.SpinSem(n=1, broken="post_no_inc"), 2, 2, "final state"),
    ("spin_sem_full_zero", mc.SpinSem(n=1, broken="full_zero"), 2, 1, "completion"),
    # Tree barrier: a node never reset, and a leaf's last arriver that releases the grid.
    ("tree_no_reset", mc.TreeBarrier(fan=2, broken="no_reset"), 3, 2, "final state"),
    ("tree_release_at_leaf", mc.TreeBarrier(fan=2, broken="release_at_leaf"), 3, 1, "passed round"),
    # Counting tree: the wrong arrival climbs (the first of a node's crossing, not the one that
    # completes it), and a root target one short.
    ("tree_count_first_climbs", mc.TreeCountBarrier(fan=2, broken="first_climbs"), 4, 2, "passed round"),
    ("tree_count_target_short", mc.TreeCountBarrier(fan=2, broken="target_short"), 3, 1, "passed round"),
    # Cluster barrier: a leader that counts in before its cluster has arrived, and every block
    # counting in globally.
    ("cluster_leader_early", mc.ClusterBarrier(c=2, broken="leader_early"), 4, 1, "passed round"),
    ("cluster_all_count", mc.ClusterBarrier(c=2, broken="all_count"), 4, 1, "passed round"),
    # Counting form of the cluster barrier: a target one short, and blocks that skip the second
    # cluster barrier that is meant to hold them until their leader saw the crossing complete.
    ("cluster_count_off_by_one", mc.ClusterCountBarrier(c=2, broken="off_by_one"), 4, 1, "passed round"),
    ("cluster_count_second_off_by_one", mc.ClusterCountBarrier(c=2, release="cluster", broken="off_by_one"), 4, 1,
     "passed round"),
    ("cluster_count_no_second", mc.ClusterCountBarrier(c=2, release="cluster", broken="no_second"), 4, 1,
     "passed round"),
]


@pytest.mark.parametrize("name,model,nproc,ops,msg", BROKEN, ids=[b[0] for b in BROKEN])
def test_planted_mistake_is_caught(name, model, nproc, ops, msg):
    r = mc.check(model, nproc, ops)
    assert not r.ok
    assert msg in r.violation


def test_queue_lock_rejects_ring_smaller_than_waiters():
    # Q must be at least the number of blocks that can wait at once.
    with pytest.raises(AssertionError):
        mc.QueueMutex(q=2).init(3, 1)


def test_wrap_safe_compare():
    assert mc.s_gt(0, 2 ** 32 - 1)
    assert not mc.s_gt(2 ** 32 - 1, 0)
    assert mc.s_ge(5, 5) and not mc.s_gt(5, 5)
