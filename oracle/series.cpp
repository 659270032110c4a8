// Numeric MapReduce oracle (the paper's Sec. 4.2): the sums
//   S(n) = sum_{i=1}^{n} sqrt(i)              (series 0)
//   A(n) = sum_{i=1}^{n} (-1)^(i+1) / i       (series 1, which tends to ln 2)
// with each term computed in IEEE double precision (the paper's Julia code
// maps integers to Float64), summed left to right in double precision with
// Neumaier's compensated summation (Neumaier 1974), so that the rounding of
// the summation itself stays near one unit in the last place.  TEST
// INFRASTRUCTURE ONLY: used by the tests and by the benchmark's CPU
// baseline, never by the product path; it shares no code with the CUDA
// library.  Pinned in tests/test_oracle_pins.py against exact rational sums,
// an exactly rounded sum (math.fsum), the Euler-Maclaurin expansion of S(n)
// and the alternating-series bound |A(n) - ln 2| < 1/(n+1).
#include <cmath>
#include <cstdint>

extern "C" {

// The series value for 0 <= n; returns 0 for series other than 0 and 1.
double oracle_series_sum(int series, uint64_t n) {
    double sum = 0.0, comp = 0.0;
    for (uint64_t i = 1; i <= n; i++) {
        double term;
        if (series == 0) {
            term = std::sqrt((double)i);
        } else if (series == 1) {
            term = 1.0 / (double)i;
            if (i % 2 == 0) term = -term;
        } else {
            return 0.0;
        }
        const double t = sum + term;
        if (std::fabs(sum) >= std::fabs(term)) comp += (sum - t) + term;
        else comp += (term - t) + sum;
        sum = t;
    }
    return sum + comp;
}

}  // extern "C"
