"""B300-native semismooth Newton solver for the continuous quadratic knapsack problem."""
