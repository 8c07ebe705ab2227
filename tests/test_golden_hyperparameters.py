"""The default workload follows the paper's hyperparameter table (App. B.3)."""

import json
import os

from paper_2408_11052_gb300 import workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hyperparameters.json")


def test_default_workload_matches_paper_table():
    h = json.load(open(GOLDEN))
    for w in (workload.SMALL_FP32, workload.ANT_AUTOGRAD):
        assert w.B == h["batch_size"]
        assert w.gamma == h["discounting"]
        assert w.lr_actor == h["policy_lr"] and w.lr_critic == h["critic_lr"]
        assert w.beta == h["logsumexp_penalty"]
        assert [w.hidden] * w.layers == h["hidden_layers"]
        assert w.repr == h["representation_dimension"]
        assert (w.energy, w.loss) == ("l2", "sym") and h["energy_function"] == "L2"
        assert w.T == h["episode_length"]
    assert workload.ANT_AUTOGRAD.E == h["num_envs"]
