"""GB300-native (sm_103a) mixed-precision ADER-DG hot path (arXiv 2504.06889)."""
