"""Run the oracle pins against the oracle library named by ORACLE_LIB; exit
0 as soon as one pin fails (the planted mistake is caught), 1 if all pass."""
import os
import sys
import tempfile

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import test_oracle_pins as T  # noqa: E402

PINS = [
    T.test_philox_known_answers,
    lambda: T.test_temperature_grid_is_uniform_with_both_ends(12, 0.2, 1.6),
    T.test_energy_closed_forms_and_symmetries,
    T.test_enumeration_closed_forms,
    T.test_pair_observables_closed_forms,
    T.test_pair_moments_enumeration_agrees_with_the_enumerator,
    T.test_sweep_incremental_energy_equals_recomputed,
    T.test_sweep_is_gauge_covariant,
    T.test_micsa_walker_leaves_the_boltzmann_weight_stationary,
    T.test_micsa_sweep_incremental_energy_equals_recomputed,
    lambda: T.test_cc_labels_match_scipy(4),
    T.test_acu_invariants,
    T.test_er_fifo_and_round_trips,
    T.test_pt_phases_touch_disjoint_pairs,
    T.test_enumeration_fluctuation_dissipation,
    T.test_couplings_from_seed_are_standard_normal_on_grid,
    T.test_init_spins_are_fair_and_distinct_per_lattice,
    T.test_houdayer_single_flips_one_negative_cluster,
    T.test_pt_acceptance_is_min_one_exp_delta,
    T.test_sdy_identity_disorder_average_is_zero,
    lambda: T.test_pthr_chain_reproduces_exact_averages_on_2x2x2(0, 0, 1, True),
    lambda: T.test_pthr_chain_reproduces_exact_averages_on_2x2x2(1, 0, 1, True),
]

if __name__ == "__main__":
    for i, pin in enumerate(PINS):
        try:
            pin()
        except Exception as e:   # AssertionError or a crash of the broken copy
            print(f"caught by pin {i}: {type(e).__name__}")
            sys.exit(0)
    print("survived")
    sys.exit(1)
